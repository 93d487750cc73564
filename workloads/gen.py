"""Seeded synthetic workloads for batched OMP.

The model is the paper's problem statement (Sec. 1): y = A x + noise, with A an M x N dictionary
(M << N) and x an s-sparse vector. Everything is drawn with NumPy's PCG64 in FP64 and rounded to
FP32 once, so every consumer (oracle, CUDA path, benchmark) sees the same FP32 inputs.

Seeding: ``SeedSequence(seed)`` is split by ``spawn_key`` into independent streams, one per
quantity (dictionary, pairing, sparsity, supports, coefficients, noise). Noise is drawn in blocks
of ``NOISE_BLOCK`` signals with a stream per block, so any slice of a batch can be regenerated
without drawing the whole batch.

The dictionary is returned as an (M, N) float32 array in Fortran order, so ``A.T`` is a
C-contiguous (N, M) array: atom n is the contiguous row n of ``A.T`` (column-major A, lda = M).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

NOISE_BLOCK = 256

# stream ids inside one SeedSequence
_S_DICT, _S_PAIR, _S_SPARSITY, _S_SUPPORT, _S_COEF, _S_NOISE, _S_TRAIN = range(7)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic OMP workload. ``sigma`` is the noise standard deviation (the configs write
    the noise as N(0, v) with v the variance, so sigma = sqrt(v))."""

    name: str
    M: int
    N: int
    B: int
    S: int                       # maximum number of OMP iterations
    s_min: int                   # planted sparsity is uniform on [s_min, s_max] (inclusive)
    s_max: int
    dict_kind: str = "gaussian"  # "gaussian" | "coherent"
    coef_kind: str = "normal"    # "normal" | "signed_uniform" | "abs_normal" (|N(0,1)|)
    sigma: float = 0.0
    eps: float = 0.0             # stop when ||r|| <= eps * ||y|| (relative form)
    precision: str = "fp32"      # correlation precision of the form this workload exercises
    coherence: float = 0.3       # coherent dictionary: squared weight of the shared component
    col_scale: float = 1.0       # Gaussian entries are drawn N(0, col_scale^2) before normalising
    group: int = 1               # supports are unions of blocks of `group` consecutive atoms
                                 # (block starts uniform without replacement); 1: plain atoms


CONFIGS = {
    # plain OMP FP32 on a small Gaussian dictionary (noiseless, fixed 8 iterations)
    "gaussian_64x256_s8_b16": Workload(
        "gaussian_64x256_s8_b16", M=64, N=256, B=16, S=8, s_min=8, s_max=8,
        sigma=0.0, precision="fp32", col_scale=1.0 / 8.0),
    # precision workload: FP32 vs BF16 correlation with FP32 top-8 rescoring
    "gaussian_1024x8192_s32_b4096": Workload(
        "gaussian_1024x8192_s32_b4096", M=1024, N=8192, B=4096, S=32, s_min=32, s_max=32,
        sigma=1e-3, precision="bf16"),
    # uneven batching: per-signal sparsity in [4, 128], relative eps stop
    "gaussian_2048x16384_s4to128_b8192": Workload(
        "gaussian_2048x16384_s4to128_b8192", M=2048, N=16384, B=8192, S=128, s_min=4,
        s_max=128, sigma=1e-3, eps=1e-3, precision="bf16"),
    # the same with a noise floor low enough for the eps stop to fire near k = s
    "gaussian_2048x16384_s4to128_b8192_lownoise": Workload(
        "gaussian_2048x16384_s4to128_b8192_lownoise", M=2048, N=16384, B=8192, S=128,
        s_min=4, s_max=128, sigma=1e-6, eps=1e-3, precision="bf16"),
    # coherent dictionary, FP8 E4M3 correlation with per-column scales
    "coherent_4096x32768_s64_b16384": Workload(
        "coherent_4096x32768_s64_b16384", M=4096, N=32768, B=16384, S=64, s_min=64,
        s_max=64, dict_kind="coherent", coef_kind="signed_uniform", sigma=1e-2,
        precision="fp8"),
    # learned-proposal evaluation batch
    "gaussian_1024x8192_s48_b16384": Workload(
        "gaussian_1024x8192_s48_b16384", M=1024, N=8192, B=16384, S=48, s_min=48, s_max=48,
        sigma=1e-3, precision="bf16"),
    # the learned-proposal workload with a support prior a network can learn: supports are 12
    # blocks of 4 consecutive atoms, coefficients |N(0,1)| (nonnegative sparse coding)
    "grouped_1024x8192_s48_g4_b16384": Workload(
        "grouped_1024x8192_s48_g4_b16384", M=1024, N=8192, B=16384, S=48, s_min=48, s_max=48,
        sigma=1e-3, precision="bf16", group=4, coef_kind="abs_normal"),
    # the paper's three application shapes (Table tab:realistic), filled with synthetic data
    "patches_256x1024_s32_b5000": Workload(
        "patches_256x1024_s32_b5000", M=256, N=1024, B=5000, S=32, s_min=32, s_max=32,
        sigma=1e-3, precision="bf16"),
    "face_8064x1207_s30_b1200": Workload(
        "face_8064x1207_s30_b1200", M=8064, N=1207, B=1200, S=30, s_min=30, s_max=30,
        sigma=1e-3, precision="bf16"),
    "audio_512x2048_s64_b5000": Workload(
        "audio_512x2048_s64_b5000", M=512, N=2048, B=5000, S=64, s_min=64, s_max=64,
        sigma=1e-3, precision="bf16"),
}


def get_config(name: str, **overrides) -> Workload:
    w = CONFIGS[name]
    return dataclasses.replace(w, **overrides) if overrides else w


def _rng(seed: int, *key: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(seed, spawn_key=tuple(key)))


def dictionary(w: Workload, seed: int = 0) -> np.ndarray:
    """Return A (M x N, float32, Fortran order) with unit-norm columns (normalised in FP64).

    "coherent": the columns are paired by a seeded random perfect matching; both columns of a
    pair share one Gaussian vector h, a_n = normalise(sqrt(1-c) g_n + sqrt(c) h), c = 0.3, so
    paired atoms have an expected inner product of about c.
    """
    rng = _rng(seed, _S_DICT)
    # draw atom by atom (rows of A^T) so the stream does not depend on the memory order
    G = rng.standard_normal((w.N, w.M)) * w.col_scale
    if w.dict_kind == "coherent":
        if w.N % 2:
            raise ValueError("coherent dictionary needs an even number of atoms")
        prng = _rng(seed, _S_PAIR)
        perm = prng.permutation(w.N)
        H = prng.standard_normal((w.N // 2, w.M))
        mate = np.empty(w.N, dtype=np.int64)
        mate[perm] = np.repeat(np.arange(w.N // 2), 2)
        G = np.sqrt(1.0 - w.coherence) * G + np.sqrt(w.coherence) * H[mate]
    elif w.dict_kind != "gaussian":
        raise ValueError(w.dict_kind)
    G /= np.sqrt(np.einsum("nm,nm->n", G, G))[:, None]
    At = np.ascontiguousarray(G, dtype=np.float32)   # (N, M), atom rows
    return At.T                                      # (M, N) view in Fortran order


def planted(w: Workload, seed: int = 0):
    """Planted supports and coefficients for the whole batch.

    Returns (sparsity[B] int32, support[B, s_max] int64 padded with -1, coef[B, s_max] float64
    padded with 0). Supports are uniform without replacement over the N atoms, or, with
    ``group`` g > 1, s / g blocks of g consecutive atoms chosen uniformly without replacement
    among the N / g blocks (a support prior a proposal network can learn).
    """
    g = _check_group(w)
    if w.s_min == w.s_max:
        sp = np.full(w.B, w.s_max, dtype=np.int32)
    else:
        sp = _rng(seed, _S_SPARSITY).integers(w.s_min, w.s_max + 1, size=w.B).astype(np.int32)
    srng = _rng(seed, _S_SUPPORT)
    sup = np.full((w.B, w.s_max), -1, dtype=np.int64)
    for b in range(w.B):
        if g == 1:
            sup[b, : sp[b]] = srng.choice(w.N, size=int(sp[b]), replace=False)
        else:
            blocks = srng.choice(w.N // g, size=int(sp[b]) // g, replace=False)
            sup[b, : sp[b]] = (blocks[:, None] * g + np.arange(g)).reshape(-1)
    crng = _rng(seed, _S_COEF)
    if w.coef_kind == "normal":
        coef = crng.standard_normal((w.B, w.s_max))
    elif w.coef_kind == "signed_uniform":
        mag = crng.uniform(0.5, 1.0, size=(w.B, w.s_max))
        sign = np.where(crng.integers(0, 2, size=(w.B, w.s_max)) == 0, -1.0, 1.0)
        coef = mag * sign
    elif w.coef_kind == "abs_normal":
        coef = np.abs(crng.standard_normal((w.B, w.s_max)))
    else:
        raise ValueError(w.coef_kind)
    coef[np.arange(w.s_max)[None, :] >= sp[:, None]] = 0.0
    return sp, sup, coef


def _check_group(w: Workload) -> int:
    g = int(w.group)
    if g < 1 or w.N % g or w.s_min % g or w.s_max % g:
        raise ValueError("group must divide N and the sparsities")
    return g


def _noise_rows(w: Workload, seed: int, lo: int, hi: int) -> np.ndarray:
    out = np.zeros((hi - lo, w.M))
    if w.sigma == 0.0:
        return out
    for blk in range(lo // NOISE_BLOCK, (hi - 1) // NOISE_BLOCK + 1):
        b0 = blk * NOISE_BLOCK
        nb = min(NOISE_BLOCK, w.B - b0)
        z = _rng(seed, _S_NOISE, blk).standard_normal((nb, w.M)) * w.sigma
        a, b = max(lo, b0), min(hi, b0 + nb)
        out[a - lo: b - lo] = z[a - b0: b - b0]
    return out


def _synthesise(A: np.ndarray, sup: np.ndarray, coef: np.ndarray, noise: np.ndarray):
    """y_b = A[:, sup_b] coef_b + noise_b in FP64 on the FP32 dictionary, rounded to FP32."""
    At64 = np.asarray(A.T, dtype=np.float64)          # (N, M)
    Y = noise.copy()
    chunk = 64
    for c0 in range(0, sup.shape[0], chunk):
        s = sup[c0: c0 + chunk]
        x = coef[c0: c0 + chunk]
        valid = s >= 0
        idx = np.where(valid, s, 0)
        cols = At64[idx]                               # (c, s_max, M)
        Y[c0: c0 + chunk] += np.einsum("csm,cs->cm", cols, np.where(valid, x, 0.0))
    return np.ascontiguousarray(Y, dtype=np.float32)


def signals(w: Workload, A: np.ndarray, seed: int = 0, rows: Optional[slice] = None):
    """Measurements Y (rows x M float32, C order) for the batch rows ``rows`` (default: all).

    Returns (Y, sparsity, support, coef) restricted to those rows. Row b is the same whichever
    slice it is drawn in.
    """
    sp, sup, coef = planted(w, seed)
    r = rows if rows is not None else slice(0, w.B)
    lo, hi, _ = r.indices(w.B)
    Y = _synthesise(A, sup[lo:hi], coef[lo:hi], _noise_rows(w, seed, lo, hi))
    return Y, sp[lo:hi], sup[lo:hi], coef[lo:hi]


def training_batch(w: Workload, n: int, chunk_id: int, seed: int = 0):
    """A chunk of training signals drawn like ``w``'s batch from streams of their own (keyed by
    ``chunk_id``), so training data never overlaps the evaluation batch. Vectorised for large
    training sets; the measurements are formed from these by ``synthesize`` (host) or on the
    device (omp_synthesize_signals).

    Returns (support int32 n x s_max (-1 padded), coef float32 n x s_max, noise float32 n x M).
    Supports are uniform without replacement: the first s distinct values of a row of uniform
    draws, which is a uniform random s-subset in random order (of blocks of ``group`` consecutive
    atoms when group > 1)."""
    rng = _rng(seed, _S_TRAIN, chunk_id)
    g = _check_group(w)
    s_max = w.s_max
    if w.s_min == w.s_max:
        sp = np.full(n, s_max, dtype=np.int32)
    else:
        sp = rng.integers(w.s_min // g, w.s_max // g + 1, size=n).astype(np.int32) * g
    nb, s_b = w.N // g, s_max // g      # draw blocks (atoms when g = 1)
    m = s_b + 32
    draws = rng.integers(0, nb, size=(n, m))
    order = np.argsort(draws, axis=1, kind="stable")
    srt = np.take_along_axis(draws, order, axis=1)
    dup_sorted = np.zeros_like(srt, dtype=bool)
    dup_sorted[:, 1:] = srt[:, 1:] == srt[:, :-1]
    dup = np.zeros_like(dup_sorted)
    np.put_along_axis(dup, order, dup_sorted, axis=1)
    keep = ~dup
    rank = np.cumsum(keep, axis=1)
    if np.any(rank[:, -1] < s_b):
        raise RuntimeError("too many repeated draws; enlarge the draw width")
    sel = keep & (rank <= s_b)
    blocks = draws[sel].reshape(n, s_b)
    sup = (blocks[:, :, None] * g + np.arange(g)).reshape(n, s_max).astype(np.int32)
    sup[np.arange(s_max)[None, :] >= sp[:, None]] = -1
    if w.coef_kind == "normal":
        coef = rng.standard_normal((n, s_max), dtype=np.float32)
    elif w.coef_kind == "abs_normal":
        coef = np.abs(rng.standard_normal((n, s_max), dtype=np.float32))
    else:
        coef = rng.uniform(0.5, 1.0, size=(n, s_max)).astype(np.float32)
        coef *= np.where(rng.integers(0, 2, size=coef.shape) == 0, -1.0, 1.0).astype(np.float32)
    coef[sup < 0] = 0.0
    if w.sigma:
        noise = rng.standard_normal((n, w.M), dtype=np.float32) * np.float32(w.sigma)
    else:
        noise = np.zeros((n, w.M), dtype=np.float32)
    return sup, coef, noise


def synthesize(A: np.ndarray, sup: np.ndarray, coef: np.ndarray, noise: np.ndarray):
    """y = A[:, sup] coef + noise per row, in FP64 on the FP32 dictionary, rounded to FP32."""
    return _synthesise(A, sup.astype(np.int64), coef.astype(np.float64), noise.astype(np.float64))
