"""Pins for oracle.gaussian: Table 1 (Sec. 3.2), alpha_Y, Philox4x32-10."""
import json
import os

import numpy as np
import pytest
from scipy import stats

from oracle import gaussian as G
from oracle.lowp import FP8_E4M3, FP8_E5M2, FP16, BF16, TF32, FP32, round_rn

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))
FMTS = {"fp8_e4m3": FP8_E4M3, "fp8_e5m2": FP8_E5M2, "fp16": FP16, "bf16": BF16,
        "tf32": TF32, "fp32": FP32}


def one_sig(x):
    return float(f"{x:.0e}")


@pytest.mark.parametrize("name", ["fp8_e4m3", "fp8_e5m2", "fp16", "bf16", "tf32"])
def test_table1_counts_by_enumeration(name):
    fmt = FMTS[name]
    for s, want in zip(GOLD["counts_s"], GOLD["counts_within_2s_sigma"][name]):
        assert G.count_within(fmt, s) == want
        assert G.count_within_formula(fmt, s) == want


def test_table1_counts_fp32_by_bit_order():
    # positive finite floats are ordered like their bit patterns, so the number
    # of values in (-2^s, 2^s) is 2 * (bits(2^s) - 1) + 1
    for s, want in zip(GOLD["counts_s"], GOLD["counts_within_2s_sigma"]["fp32"]):
        b = int(np.array(2.0 ** s, dtype=np.float32).view(np.uint32))
        assert 2 * (b - 1) + 1 == want
        assert G.count_within_formula(FP32, s) == want


@pytest.mark.parametrize("name", ["fp8_e4m3", "fp8_e5m2", "fp16"])
def test_table1_probabilities(name):
    fmt = FMTS[name]
    assert one_sig(G.p_not_normalized(fmt)) == GOLD["p_not_normalized"][name]
    assert one_sig(G.p_underflow(fmt)) == GOLD["p_underflow"][name]
    assert G.p_overflow(fmt) < GOLD["p_overflow_upper_bound"]


def test_table1_wide_exponent_formats():
    for fmt in (BF16, TF32, FP32):
        assert G.p_not_normalized(fmt) < GOLD["p_wide_exponent_upper_bound"]
        assert G.p_overflow(fmt) < GOLD["p_overflow_upper_bound"]


def test_underflow_probability_monte_carlo_e4m3():
    rng = np.random.default_rng(11)
    g = rng.standard_normal(4_000_000)
    frac = np.mean(round_rn(g, FP8_E4M3) == 0)
    p = G.p_underflow(FP8_E4M3)
    assert abs(frac - p) < 5 * np.sqrt(p / g.size)


@pytest.mark.parametrize("fmt", [FP8_E4M3, FP8_E5M2, FP16])
def test_alpha_Y_matches_monte_carlo(fmt):
    rng = np.random.default_rng(3)
    g = rng.standard_normal(4_000_000)
    r = round_rn(g, fmt)
    var = np.mean(r * r)
    a = G.alpha_Y(fmt)
    se = np.std(r * r) / np.sqrt(g.size)
    assert abs(var - a) < 5 * se


def test_alpha_Y_approaches_one_with_mantissa():
    devs = [abs(G.alpha_Y(f) - 1.0) for f in (FP8_E5M2, FP8_E4M3, BF16, FP16)]
    # mantissa lengths 2, 3, 7, 10: the deviation shrinks with Y
    assert devs[0] > devs[1] > devs[2] > devs[3]
    assert devs[3] < 1e-6
    # uniform-rounding-error approximation alpha ~ 1 + E[q^2]/12 for FP16
    assert abs(G.alpha_Y(FP16) - 1.0) < (2.0 ** -10) ** 2


def test_philox_known_answers():
    # Random123 known-answer vectors for philox4x32_10
    out = G.philox4x32_10([0, 0, 0, 0], [0, 0])
    assert [int(v) for v in out] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    out = G.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2)
    assert [int(v) for v in out] == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    out = G.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                          [0xA4093822, 0x299F31D0])
    assert [int(v) for v in out] == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_gaussian_stream_is_standard_normal():
    z = G.gaussian_f64(seed=42, offset=0, rows=1000, cols=257).ravel()
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_gaussian_stream_layout_and_offset():
    a = G.gaussian_f64(seed=9, offset=0, rows=8, cols=6).ravel()
    b = G.gaussian_f64(seed=9, offset=3, rows=2, cols=6).ravel()     # 3 blocks = 12 elements later
    assert np.array_equal(a[12:24], b)
    c = G.gaussian_f64(seed=10, offset=0, rows=8, cols=6).ravel()
    assert not np.allclose(a, c)


def test_box_muller_inverse_map():
    # Box-Muller maps (u1, u2) to polar coordinates: radius^2 = -2 ln u1 and
    # angle = 2 pi u2.  Invert the output with exp and atan2 (not the
    # forward formula) and recover the inputs: a swapped cos / sin, a
    # missing factor 2 or a wrong logarithm changes them.
    rng = np.random.default_rng(3)
    u1 = rng.uniform(1e-9, 1.0, size=20000)
    u2 = rng.uniform(0.0, 1.0, size=20000)
    z0, z1 = G.box_muller(u1, u2)
    assert np.allclose(np.exp(-(z0 * z0 + z1 * z1) / 2.0), u1, rtol=1e-12, atol=0)
    ang = np.mod(np.arctan2(z1, z0) / (2.0 * np.pi), 1.0)
    d = np.abs(ang - u2)
    assert np.all(np.minimum(d, 1.0 - d) < 1e-12)
    # fixed points: u2 = 0 puts the whole radius on z0, u2 = 1/4 on z1
    r = np.sqrt(-2.0 * np.log(0.25))
    a, b = G.box_muller(np.array([0.25]), np.array([0.0]))
    assert a[0] == pytest.approx(r, rel=1e-15) and abs(b[0]) < 1e-15
    a, b = G.box_muller(np.array([0.25]), np.array([0.25]))
    assert abs(a[0]) < 1e-15 and b[0] == pytest.approx(r, rel=1e-15)


def test_gaussian_stream_quantiles():
    # empirical quantiles of 10^6 draws of the stream against the normal
    # quantile function (scipy's ndtri, independent of the Box-Muller code);
    # the standard error of the q-quantile is sqrt(q (1 - q) / n) / phi(x_q)
    from scipy.special import ndtri
    z = np.sort(G.gaussian_f64(seed=77, offset=0, rows=1000, cols=1000).ravel())
    n = z.size
    for q in (0.001, 0.01, 0.1, 0.25, 0.5, 0.75, 0.9, 0.99, 0.999):
        xq = float(ndtri(q))
        se = np.sqrt(q * (1 - q) / n) / (np.exp(-xq * xq / 2) / np.sqrt(2 * np.pi))
        assert abs(z[int(q * n)] - xq) < 5 * se, (q, z[int(q * n)], xq, se)
    # both outputs of a pair are standard normal and uncorrelated
    zz = G.gaussian_f64(seed=78, offset=0, rows=250000, cols=4)
    c = np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]
    assert abs(c) < 5 / np.sqrt(zz.shape[0])


def test_gaussian_f16_is_the_half_rounding_of_the_stream():
    # gaussian_f16 rounds the float64 stream RN-even to FP16: numpy's
    # double -> half cast is an independent correctly rounded conversion
    x = G.gaussian_f64(123, 7, 64, 97)
    h = G.gaussian_f16(123, 7, 64, 97)
    assert h.shape == (64, 97)
    assert np.array_equal(h, x.astype(np.float16).astype(np.float64))
    assert np.array_equal(round_rn(h, FP16), h)
    assert np.all(np.abs(h - x) <= FP16.u * np.abs(x) + FP16.min_subnormal)
