"""Error bounds of the two FP32-for-FP64 substitutions in the update and Gram-space kernels,
restated here in IEEE FP32 arithmetic (numpy float32, round to nearest even, no contraction):

  * ||z||^2 as an unevaluated sum hi + lo of FP32 numbers: each square split exactly by an FMA
    (p = fl(z*z), e = z*z - p exactly), partial sums combined with Knuth's two-sum; the kernels
    claim about 2^-42 relative for the sums they form (up to 64 terms per thread, 32 lanes, 8
    warps);
  * gamma = 1/sqrt(delta) from an FP32 reciprocal square root seed (CUDA documents rsqrtf to
    within 2 ulp) and one Newton-Raphson step y (3 - delta y^2) / 2 in FP64: the relative error
    squares: about 2^-42 relative with the seed 2 ulp off and delta rounded to FP32.

A plain FP32 sum of the same squares misses the first bound by orders of magnitude, so the test
would catch a lost error term."""
import math

import numpy as np

f32 = np.float32


def two_sum(s, e, x):
    t = f32(s + x)
    xv = f32(t - s)
    err = f32(f32(s - f32(t - xv)) + f32(x - xv))
    return t, f32(e + err)


def exact_square_split(z):
    p = f32(z * z)
    # the FMA residual z*z - p is exact: compute it exactly in FP64 (z*z is exact there) and round
    e = f32(np.float64(z) * np.float64(z) - np.float64(p))
    assert np.float64(e) == np.float64(z) * np.float64(z) - np.float64(p)
    return p, e


def double_float_sum_of_squares(zs, lanes=32):
    """Per-lane accumulation, then a butterfly over the lanes, as the kernels do."""
    hi = [f32(0)] * lanes
    lo = [f32(0)] * lanes
    for j, z in enumerate(zs):
        l = j % lanes
        p, e = exact_square_split(f32(z))
        lo[l] = f32(lo[l] + e)
        hi[l], lo[l] = two_sum(hi[l], lo[l], p)
    o = lanes // 2
    while o:
        nh, nl = list(hi), list(lo)
        for l in range(lanes):
            m = l ^ o
            nl[l] = f32(lo[l] + lo[m])
            nh[l], nl[l] = two_sum(hi[l], nl[l], hi[m])
        hi, lo = nh, nl
        o //= 2
    return np.float64(hi[0]) + np.float64(lo[0])


def test_double_float_sum_of_squares():
    rng = np.random.default_rng(0)
    worst = 0.0
    for n in (1, 7, 31, 64, 200, 256):
        for trial in range(20):
            kind = trial % 3
            if kind == 0:
                z = rng.standard_normal(n)
            elif kind == 1:
                z = rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))
            else:
                z = 1.0 + rng.standard_normal(n) * 1e-4   # nearly equal terms (cancellation-free,
            z = z.astype(np.float32)                      # but every sum rounds)
            exact = math.fsum((z.astype(np.float64) ** 2).tolist())
            got = double_float_sum_of_squares(z)
            worst = max(worst, abs(got - exact) / exact)
    assert worst <= 2.0 ** -42
    # the plain FP32 sum of the same squares is far worse: the split is doing the work
    z = (1.0 + rng.standard_normal(256) * 1e-4).astype(np.float32)
    exact = math.fsum((z.astype(np.float64) ** 2).tolist())
    plain = np.float64(np.sum(z * z, dtype=np.float32))
    assert abs(plain - exact) / exact > 2.0 ** -30


def newton_rsqrt(delta, seed_ulps):
    """FP32 seed off by `seed_ulps` ulp (CUDA's rsqrtf bound is 2), then one FP64 step."""
    y32 = f32(1.0 / math.sqrt(float(f32(delta))))
    y32 = np.nextafter(y32, f32(np.inf) if seed_ulps > 0 else f32(0), dtype=np.float32) \
        if seed_ulps else y32
    for _ in range(abs(seed_ulps) - 1):
        y32 = np.nextafter(y32, f32(np.inf) if seed_ulps > 0 else f32(0), dtype=np.float32)
    y0 = np.float64(y32)
    return y0 * (1.5 - 0.5 * delta * y0 * y0)


def test_newton_reciprocal_square_root():
    rng = np.random.default_rng(1)
    deltas = np.concatenate([np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 400)),
                             [1e-35, 3.7e-20, 1.0, 2.0, 0.5, 1e35]])
    worst = 0.0
    for d in deltas:
        ref = 1.0 / math.sqrt(d)
        for ulps in (-2, -1, 0, 1, 2):
            worst = max(worst, abs(newton_rsqrt(d, ulps) - ref) / ref)
    assert worst <= 2.0 ** -42
