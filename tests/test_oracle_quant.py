"""Pins for the oracle's BF16 / FP8 E4M3 rounding: the formats' own definitions (code tables,
exact midpoints), and PyTorch's CPU conversions as an independent library routine."""
import numpy as np
import torch

from oracle import quant


def _halfway_bf16_inputs():
    # x exactly halfway between two BF16 neighbours: low 16 bits = 0x8000
    hi = np.arange(0x3F80, 0x3F80 + 64, dtype=np.uint32)
    return ((hi << 16) | 0x8000).view(np.float32)


def test_bf16_ties_to_even():
    x = _halfway_bf16_inputs()
    out = quant.bf16_round(x).view(np.uint32) >> 16
    hi = x.view(np.uint32) >> 16
    want = np.where(hi % 2 == 0, hi, hi + 1)
    assert np.array_equal(out, want)


def test_bf16_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([
        (rng.standard_normal(200000) * 10.0 ** rng.integers(-30, 30, 200000)).astype(np.float32),
        _halfway_bf16_inputs(),
        np.array([0.0, -0.0, 1e-45, -1e-45, 3.4e38, -3.4e38, np.inf, -np.inf], np.float32),
    ])
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    got = quant.bf16_round(x)
    assert np.array_equal(ref.view(np.uint32), got.view(np.uint32))


def test_e4m3_table_definition():
    """126 finite positive codes + zero; max 448 = 1.75 * 2^8; min subnormal 2^-9; min normal
    2^-6; values strictly increase with the code."""
    v = quant.E4M3_VALUES
    assert v.size == 127 and v[0] == 0 and v[1] == 2.0 ** -9 and v[8] == 2.0 ** -6
    assert v[-1] == 448.0 and np.all(np.diff(v) > 0)
    codes = np.arange(256, dtype=np.uint8)
    vals = quant.e4m3_value(codes)
    finite = ~np.isnan(vals)
    assert np.sum(~finite) == 2                                  # 0x7F and 0xFF
    back = quant.e4m3_code(vals[finite].astype(np.float32))
    assert np.array_equal(back, codes[finite])                    # exact values round-trip


def test_e4m3_midpoints_and_saturation():
    v = quant.E4M3_VALUES
    mids = ((v[:-1] + v[1:]) / 2).astype(np.float32)
    assert np.all(mids.astype(np.float64) == (v[:-1] + v[1:]) / 2)  # midpoints exact in FP32
    codes = quant.e4m3_code(mids)
    lo = np.arange(126)
    want = np.where(lo % 2 == 0, lo, lo + 1)
    assert np.array_equal(codes, want.astype(np.uint8))
    big = np.array([448.0, 449.0, 464.0, 500.0, 1e30, np.inf, -1e9, -np.inf], np.float32)
    assert np.array_equal(quant.e4m3_value(quant.e4m3_code(big)),
                          [448, 448, 448, 448, 448, 448, -448, -448])
    assert np.isnan(quant.e4m3_value(quant.e4m3_code(np.array([np.nan], np.float32))))[0]


def test_e4m3_matches_torch_in_range():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(200000) * 10.0 ** rng.uniform(-4, 2.6, 200000)).astype(np.float32)
    x = np.clip(x, -448, 448)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ref, quant.e4m3_code(x))


def test_fp8_scale_rows_error_bound():
    """Per-row scaling: the largest |entry| maps to 448 exactly (up to FP32 rounding of the
    scale) and every decoded entry is within half an E4M3 ulp (relative 2^-4) of x, or within
    the subnormal step near 0."""
    rng = np.random.default_rng(2)
    X = (rng.standard_normal((64, 300)) * rng.uniform(0.01, 10, size=(64, 1))).astype(np.float32)
    X[3] = 0.0
    codes, scale = quant.fp8_scale_rows(X)
    assert scale[3] == 0 and np.all(codes[3] == 0)
    dec = quant.e4m3_value(codes) * scale[:, None].astype(np.float64)
    err = np.abs(dec - X)
    bound = np.maximum(np.abs(X) * 2.0 ** -4, scale[:, None] * 2.0 ** -10) * 1.0001
    assert np.all(err <= bound)
    amax_codes = codes[np.arange(64), np.argmax(np.abs(X), axis=1)] & 0x7F
    assert np.all((amax_codes == 0x7E) | (scale == 0))
