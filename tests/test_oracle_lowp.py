"""Pins for oracle.lowp: RN-even rounding to eXmY formats (Sec. 3.1).

Independent references: numpy's float32->float16 cast, torch's
float32->bfloat16 cast (both RN-even), exhaustive FP16 bit patterns, and
hand-placed ties.
"""
import numpy as np
import pytest
import torch

from oracle.lowp import FP16, BF16, FP8_E4M3, round_rn, decode_bits, all_finite_values


def test_decode_all_fp16_patterns_matches_numpy():
    bits = np.arange(1 << 16, dtype=np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    got = decode_bits(bits.astype(np.int64), FP16)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.array_equal(got[np.isinf(ref)], ref[np.isinf(ref)])


def test_fp16_roundtrip_every_value():
    v = all_finite_values(FP16)
    assert np.array_equal(round_rn(v, FP16), v)


def test_fp16_ties_go_to_even():
    v = np.unique(all_finite_values(FP16))
    mids = 0.5 * (v[1:] + v[:-1])               # exact midpoints (fit in float64)
    got = round_rn(mids, FP16)
    ref = mids.astype(np.float32).astype(np.float16).astype(np.float64)
    assert np.array_equal(got, ref)
    # even = last mantissa bit zero
    bits = got.astype(np.float16).view(np.uint16)
    assert np.all((bits & 1) == 0)


def test_fp16_random_fp32_values_match_numpy():
    rng = np.random.default_rng(123)
    x = np.concatenate([
        rng.standard_normal(200_000).astype(np.float32),
        (rng.standard_normal(100_000) * 1e-5).astype(np.float32),     # subnormal range
        (rng.uniform(-1, 1, 100_000) * 70000).astype(np.float32),     # overflow range
    ])
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    got = round_rn(x.astype(np.float64), FP16)
    assert np.array_equal(got, ref)


def test_fp16_overflow_threshold():
    # 65504 is max; 65520 is the midpoint to 2^16 and rounds to even (inf).
    got = round_rn(np.array([65504.0, 65519.99609375, 65520.0, -65520.0]), FP16)
    assert got[0] == 65504.0 and got[1] == 65504.0
    assert np.isinf(got[2]) and got[3] == -np.inf


def test_bf16_matches_torch_cast():
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(100_000), rng.standard_normal(10_000) * 1e-39]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = round_rn(x.astype(np.float64), BF16)
    assert np.array_equal(got, ref)


def test_fp8_e4m3_values():
    v = np.unique(all_finite_values(FP8_E4M3))
    assert v.max() == 240.0                       # IEEE-style e4m3: (2 - 2^-3) 2^7
    assert np.min(v[v > 0]) == 2.0 ** -9          # min subnormal 2^(1-7-3)


@pytest.mark.parametrize("fmt", [FP16, BF16, FP8_E4M3])
def test_rn_error_bound(fmt):
    """|g_eXmY - g| <= exp_of(g_eXmY) * u_Y for normal results (Eq. RN-range)."""
    rng = np.random.default_rng(5)
    g = rng.standard_normal(100_000)
    r = round_rn(g, fmt)
    nz = (np.abs(r) >= fmt.min_normal) & np.isfinite(r)
    e = 2.0 ** np.floor(np.log2(np.abs(r[nz])))
    assert np.all(np.abs(r[nz] - g[nz]) <= e * fmt.u * (1 + 1e-15))


def test_f16_to_f64_bits_and_half_inputs_agree_with_numpy():
    # both input forms of f16_to_f64 (uint16 bit patterns and float16 data)
    # against numpy's own half -> double widening, over every finite pattern
    from oracle.lowp import f16_to_f64
    bits = np.arange(1 << 16, dtype=np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    fin = np.isfinite(ref)
    assert np.array_equal(f16_to_f64(bits)[fin], ref[fin])
    assert np.array_equal(f16_to_f64(bits.view(np.float16))[fin], ref[fin])
    # the sign of zero survives the bit-pattern path
    assert np.signbit(f16_to_f64(np.array([0x8000], dtype=np.uint16)))[0]


def test_bf16_decode_and_encode_against_torch():
    # every BF16 bit pattern: the decoded value equals torch's bfloat16 ->
    # float64 widening, and encoding the finite values returns the pattern
    from oracle.lowp import bf16_to_f64, encode_bf16
    bits = np.arange(1 << 16, dtype=np.uint16)
    ref = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    got = bf16_to_f64(bits)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.array_equal(got[np.isinf(ref)], ref[np.isinf(ref)])
    assert np.array_equal(encode_bf16(got[fin]), bits[fin])
