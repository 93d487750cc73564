"""BF16 and FP8 E4M3 rounding from the formats' definitions (test infrastructure only).

These decide integer outcomes (the stored codes) that the CUDA path must reproduce bit for bit,
so every step is done in the same FP32 operations the kernels use:
  bf16(x):  round-to-nearest-even to 8 significand bits, exponent range of FP32;
  e4m3(x):  OCP E4M3 ("fn": bias 7, 3 mantissa bits, max 448, no infinities, NaN = S.1111.111),
            round-to-nearest-even, saturating to +-448 ("satfinite");
  FP8 scaling: per atom s_a = amax|a_n| / 448 and a_q = e4m3(a * (448 / amax)) with the
            quotient and the product each rounded to FP32; per signal the same with amax|r_b|.
            A zero vector gets scale 0 and all-zero codes.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Nearest BF16 value (ties to even) of FP32 inputs, returned as FP32.

    BF16 keeps the upper 16 bits of an FP32 word. Rounding to nearest with ties to even adds
    half a unit of the kept part minus one, plus the kept part's lowest bit, to the discarded
    16 bits, then truncates; an overflow carries into the exponent (up to infinity), which is
    what round-to-nearest prescribes. NaNs map to the canonical quiet NaN."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).copy()
    out[np.isnan(x)] = np.float32(np.nan)
    return out


def _e4m3_table():
    """Values of the non-negative finite E4M3 codes 0x00..0x7E, in code order (increasing)."""
    vals = []
    for code in range(0x7F):
        e, m = code >> 3, code & 7
        if e == 0:
            vals.append(m / 8.0 * 2.0 ** -6)
        else:
            vals.append((1.0 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(vals)


E4M3_VALUES = _e4m3_table()


def e4m3_code(x: np.ndarray) -> np.ndarray:
    """E4M3 codes (uint8) of FP32 inputs: round to nearest, ties to the even code, saturate
    finite and infinite overflow to the largest finite magnitude; NaN -> 0x7F | sign."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    sign = np.signbit(x)
    a = np.abs(x)
    nan = np.isnan(x)
    a = np.where(nan, 0.0, np.minimum(a, E4M3_MAX))
    hi = np.searchsorted(E4M3_VALUES, a, side="left")          # first value >= a
    hi = np.minimum(hi, E4M3_VALUES.size - 1)
    lo = np.maximum(hi - 1, 0)
    dlo = a - E4M3_VALUES[lo]
    dhi = E4M3_VALUES[hi] - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    code = np.where(pick_hi, hi, lo)
    code = code.astype(np.uint8) | (sign.astype(np.uint8) << 7)
    code[nan] = 0x7F | (sign[nan].astype(np.uint8) << 7)
    return code


def e4m3_value(code: np.ndarray) -> np.ndarray:
    """FP64 value of E4M3 codes (NaN for the two NaN codes)."""
    code = np.asarray(code, dtype=np.uint8)
    mag = code & 0x7F
    v = np.where(mag == 0x7F, np.nan, E4M3_VALUES[np.minimum(mag, 0x7E)])
    return np.where(code & 0x80, -v, v)


def e4m3_round(x: np.ndarray) -> np.ndarray:
    return e4m3_value(e4m3_code(x))


def fp8_scale_rows(X: np.ndarray):
    """Per-row FP8 scaling of an FP32 matrix (rows = atoms of A^T, or signals of R).

    Returns (codes uint8 same shape, scale float32 per row) with scale = amax / 448 and
    codes = e4m3(x * (448 / amax)), every operation rounded to FP32 as the kernels do."""
    X = np.asarray(X, dtype=np.float32)
    amax = np.max(np.abs(X), axis=1).astype(np.float32)
    nz = amax > 0
    inv = np.zeros_like(amax)
    inv[nz] = (np.float32(E4M3_MAX) / amax[nz]).astype(np.float32)
    scale = np.zeros_like(amax)
    scale[nz] = (amax[nz] / np.float32(E4M3_MAX)).astype(np.float32)
    Xs = (X * inv[:, None]).astype(np.float32)
    return e4m3_code(Xs), scale
