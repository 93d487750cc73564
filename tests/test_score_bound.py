"""The score error bound of the quantised paths (omp_score_error_bound, a host-only C-ABI call)
against the formats' own rounding: on random and adversarial vectors, quantised with the
oracle's BF16 and E4M3 rounding (FP8 with the per-row amax/448 scale the kernels use), the exact
dot product of the quantised operands differs from the exact FP32 dot product by at most
bound * ||a|| * ||r||. The adversarial cases round every element the same way by almost half an
ulp, so they reach most of the bound: a bound missing a term or a factor fails them.

The skip and trim of the FP32 rescoring and the pruning of the BF16 correlation are exact only if
this bound holds (the GPU tests check the consequence: bit-identical results with the bound on
and off)."""
import math

import numpy as np
import pytest

from oracle import quant
from paper_2407_06434_gb300 import build as libbuild
from paper_2407_06434_gb300 import omp

BF16, FP8 = 1, 2


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return omp.load()


def exact_dot(x, y):
    return math.fsum((np.asarray(x, np.float64) * np.asarray(y, np.float64)).tolist())


def q_bf16(x):
    return quant.bf16_round(np.asarray(x, np.float32)).astype(np.float64)


def q_fp8(x):
    codes, scale = quant.fp8_scale_rows(np.asarray(x, np.float32)[None, :])
    return quant.e4m3_value(codes[0]) * np.float64(scale[0])


def worst_ratio(quantise, pairs):
    """max over the pairs of |q(a).q(r) - a.r| / (||a|| ||r||)"""
    worst = 0.0
    for a, r in pairs:
        a = np.asarray(a, np.float32)
        r = np.asarray(r, np.float32)
        d = abs(exact_dot(quantise(a), quantise(r)) - exact_dot(a, r))
        worst = max(worst, d / (np.linalg.norm(a.astype(np.float64)) * np.linalg.norm(r.astype(np.float64))))
    return worst


def random_pairs(M, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 3
        if kind == 0:
            a, r = rng.standard_normal(M), rng.standard_normal(M)
        elif kind == 1:  # heavy tails: a few large entries, most of the mass tiny
            a, r = rng.standard_cauchy(M), rng.standard_cauchy(M)
        else:  # wide exponent spread (many entries in E4M3's subnormal range after scaling)
            a = rng.standard_normal(M) * np.exp2(rng.integers(-20, 1, M))
            r = rng.standard_normal(M) * np.exp2(rng.integers(-20, 1, M))
        out.append((a, r))
    return out


def test_bound_values():
    assert omp.omp_score_error_bound(0, 1024) == 0.0            # FP32: no bound, always rescore
    assert omp.omp_score_error_bound(BF16, 0) == 0.0
    assert omp.omp_score_error_bound(7, 1024) == 0.0            # unknown precision
    for prec, lo in ((BF16, 2.0 ** -7), (FP8, 2.0 ** -3)):      # at least 2u
        b = [omp.omp_score_error_bound(prec, m) for m in (64, 1024, 8192)]
        assert b[0] > lo and b[0] < b[1] < b[2] < 2 * lo         # grows with Mp, stays O(u)


@pytest.mark.parametrize("M", [64, 1024, 4096])
def test_bf16_bound_holds(M):
    bound = omp.omp_score_error_bound(BF16, M)
    assert worst_ratio(q_bf16, random_pairs(M, 30, M)) <= bound
    # every element rounded down by almost half an ulp (2^-8 relative), in both operands
    x = np.full(M, 1.0 + 0.499 * 2.0 ** -7, np.float32)
    w = worst_ratio(q_bf16, [(x, x)])
    assert 0.9 * 2 * 2.0 ** -8 <= w <= bound   # reaches 2u: a bound without the 2 fails


@pytest.mark.parametrize("M", [64, 1024, 4096])
def test_fp8_bound_holds(M):
    bound = omp.omp_score_error_bound(FP8, M)
    assert worst_ratio(q_fp8, random_pairs(M, 30, 10 * M)) <= bound
    # one entry sets the scale (it maps to 448 exactly); the others sit almost half an ulp
    # (2^-4 relative) above an E4M3 value in the normal range and round down
    x = np.full(M, 1.0 + 0.499 * 2.0 ** -3, np.float32)
    x[0] = 448.0 / 256.0
    w = worst_ratio(q_fp8, [(x, x)])
    assert 0.85 * 2 * 2.0 ** -4 <= w <= bound  # about 2u/(1+u): a bound without the 2 fails


def test_fp8_subnormal_range_is_covered():
    """Entries far below the row's amax land in E4M3's subnormal range, where the rounding error
    is half the subnormal spacing of the scale rather than relative to the entry. One large entry
    sets the scale, every other entry sits just below the middle of two subnormal codes (so all
    round the same way), and the other operand is dense; the bound's sqrt(Mp) term covers it."""
    for M in (1024, 4096):
        bound = omp.omp_score_error_bound(FP8, M)
        a = np.full(M, 1.49 * 2.0 ** -9, np.float32)   # scale 1: codes 2^-9 apart down here
        a[0] = 448.0
        codes, scale = quant.fp8_scale_rows(a[None, :])
        assert scale[0] == 1.0
        sub = codes[0, 1:]
        assert np.all((sub & 0x78) == 0) and np.all((sub & 0x07) != 0)   # subnormal codes
        r = np.ones(M, np.float32)
        w = worst_ratio(q_fp8, [(a, r)])
        assert w <= bound
        # the subnormal part alone: (M - 1) errors of 0.49 2^-9 against ||a|| ||r|| ~ 448 sqrt(M)
        assert w > 0.9 * (M - 1) * 0.49 * 2.0 ** -9 / (448.0 * np.sqrt(M))


def test_running_best_window_keeps_the_pick_and_the_rescoring_window():
    """The correlation epilogue drops a column whose quantised score is at or below the best
    quantised score seen so far, less three bounds eps ||r||. Scanned in the kernel's order
    (ascending columns, the running best taken over whole 32-column chunks, this chunk's
    included), with the oracle's BF16 rounding: no dropped column is the exact argmax (lowest
    index on ties) or lies within the rescoring window, 2 eps ||r|| below the best quantised
    score. Columns are drawn near the best so that the window is crowded."""
    M, N = 1024, 4096
    eps = omp.omp_score_error_bound(BF16, M)
    rng = np.random.default_rng(7)
    for trial in range(6):
        A = rng.standard_normal((N, M)).astype(np.float32)
        r = rng.standard_normal(M).astype(np.float32)
        # crowd the top: columns that are the residual's direction plus noise of varying size,
        # so that many quantised scores fall within a few bounds of each other
        near = rng.choice(N, 64, replace=False)
        A[near] = (r[None, :] * rng.uniform(0.9, 1.0, (64, 1)) +
                   rng.standard_normal((64, M)) * rng.uniform(0.0, 0.05 * (trial + 1), (64, 1))).astype(np.float32)
        nrm = np.linalg.norm(A.astype(np.float64), axis=1)
        Aq = quant.bf16_round(A).astype(np.float64)
        rq = quant.bf16_round(r).astype(np.float64)
        exact = np.abs(A.astype(np.float64) @ r.astype(np.float64)) / nrm
        qsc = np.abs(Aq @ rq) / nrm
        rn = float(np.linalg.norm(r.astype(np.float64)))
        win3 = 3.0 * eps * rn
        chunk_best = np.maximum.accumulate(qsc.reshape(-1, 32).max(axis=1))
        dropped = qsc <= np.repeat(chunk_best, 32) - win3
        pick = int(np.argmax(exact))                  # lowest index among equal maxima
        assert not dropped[pick]
        in_window = qsc >= qsc.max() - 2.0 * eps * rn
        assert not np.any(dropped & in_window)
        assert dropped.sum() > N // 2                 # the window does prune
