"""Pins for oracle.shgemm (Sec. 4.1, 4.3, 4.4.1)."""
import numpy as np
import pytest

from oracle import shgemm as S
from oracle.lowp import FP16, round_rn
from synth import omega_f16, uniform


def test_project_exact_integer_brute_force():
    # integer-valued A and Omega: every path is exact; compare with Python ints
    rng = np.random.default_rng(0)
    A = rng.integers(-50, 50, size=(8, 8)).astype(np.float32)
    W = rng.integers(-20, 20, size=(8, 8)).astype(np.float16)
    Y = S.project_exact(A, W)
    ref = [[sum(int(A[i, l]) * int(W[l, j]) for l in range(8)) for j in range(8)] for i in range(8)]
    assert np.array_equal(Y, np.array(ref, dtype=np.float64))
    # integers below 2^11 split exactly into hi with lo = 0
    hi, lo = S.split_f16(A)
    assert np.array_equal(hi, A.astype(np.float64)) and not lo.any()


def test_project_exact_t_integer_brute_force():
    # the transposed projection A^T B (power scheme, TN products) on a
    # non-square integer case: C[i, j] = sum_r A[r, i] B[r, j] with Python
    # integers; a transposed operand or a swapped index gives another matrix
    rng = np.random.default_rng(1)
    A = rng.integers(-40, 40, size=(9, 5)).astype(np.float32)     # n x m, contracted over n
    B = rng.integers(-30, 30, size=(9, 3)).astype(np.float16)     # n x k
    C = S.project_exact_t(A, B)
    assert C.shape == (5, 3)
    ref = [[sum(int(A[r, i]) * int(B[r, j]) for r in range(9)) for j in range(3)] for i in range(5)]
    assert np.array_equal(C, np.array(ref, dtype=np.float64))
    # FP32 values that are not integers are taken exactly (24-bit significands)
    a = np.float32(1.0 + 2.0 ** -23)
    assert S.project_exact_t(np.array([[a]], np.float32), np.array([[3.0]]))[0, 0] == 3.0 * (1.0 + 2.0 ** -23)


def test_project_exact_uses_fp16_bits():
    W = omega_f16(64, 5, 1)
    A = uniform(7, 64, 2)
    assert np.array_equal(S.project_exact(A, W), S.project_exact(A, W.view(np.uint16)))


def test_split_reconstruction_and_inequalities():
    A = np.concatenate([uniform(64, 64, 3), uniform(64, 64, 4, -1e-3, 1e-3),
                        uniform(64, 64, 5, -3e4, 3e4)])
    hi, lo = S.split_f16(A)
    a = A.astype(np.float64)
    rest = a - hi - lo * 2.0 ** -11
    # Eq. split-matrix-ineq, all three
    assert S.split_bounds(A) == (True, True, True)
    # hi, lo are FP16 values
    assert np.array_equal(round_rn(hi, FP16), hi) and np.array_equal(round_rn(lo, FP16), lo)
    # the residual is tiny but usually non-zero (mantissa loss of the split)
    normal = np.abs(a) >= 2.0 ** -14
    assert np.all(np.abs(rest[normal]) <= 2.0 ** -22 * np.abs(a[normal]))
    assert np.count_nonzero(rest) > 0
    # below 2^-14 hi is subnormal and the relative bound does not apply, but
    # the absolute error stays below half an FP16-subnormal ulp of lo * 2^-11
    assert np.all(np.abs(rest[~normal]) <= 2.0 ** -25 * 2.0 ** -11 * (1 + 1e-12))


def test_split_mantissa_loss_expected_quarter_bit():
    """A_delta carries on average about 0.25 bit of a (Sec. 4.3).

    For a uniform in [1, 2): hi has 11 significant bits, lo another 11, so 2
    of a's 24 bits remain for A_delta; the measured mean information lost,
    log2(1 + |A_delta| / ulp(a)), is ~0.25 bit."""
    rng = np.random.default_rng(1)
    A = rng.uniform(1, 2, 200_000).astype(np.float32)
    hi, lo = S.split_f16(A)
    rest = A.astype(np.float64) - hi - lo * 2.0 ** -11
    ulp = 2.0 ** -23
    bits = np.log2(1.0 + np.abs(rest) / ulp)
    assert 0.1 < bits.mean() < 0.5


def test_emulated_shgemm_close_to_exact():
    A = uniform(40, 300, 6)
    W = omega_f16(300, 17, 7)
    Yx = S.project_exact(A, W)
    Ye = S.shgemm_emulated(A, W)
    # representation error only: |A_delta| |W| <= u16^2 |A| |W|
    bound = S.U_FP16 ** 2 * (np.abs(A.astype(np.float64)) @ np.abs(W.astype(np.float64)))
    assert np.all(np.abs(Ye - Yx) <= bound * (1 + 1e-12))
    assert np.any(Ye != Yx)
    # a wrong lo scale (2^-10) would break the bound by far
    hi, lo = S.split_f16(A)
    wrong = hi @ W.astype(np.float64) + lo @ W.astype(np.float64) * 2.0 ** -10
    assert np.max(np.abs(wrong - Yx) / (bound + 1e-300)) > 10


def _fp32_blocked_dot(A, W, block=8):
    """FP32 SIMT product with 8-element blocks summed in FP32, then the block
    sums accumulated sequentially in FP32 (the SIMT analogue of Sec. 4.3)."""
    A32 = A.astype(np.float32)
    W32 = W.astype(np.float32)
    m, n = A32.shape
    k = W32.shape[1]
    acc = np.zeros((m, k), dtype=np.float32)
    for b in range(0, n, block):
        t = np.zeros((m, k), dtype=np.float32)
        for l in range(b, min(n, b + block)):
            t = (t + np.outer(A32[:, l], W32[l]).astype(np.float32)).astype(np.float32)
        acc = (acc + t).astype(np.float32)
    return acc


def test_elementwise_bound_covers_fp32_blocked_sum():
    A = uniform(16, 512, 8)
    W = omega_f16(512, 8, 9)
    Yx = S.project_exact(A, W)
    Yf = _fp32_blocked_dot(A, W)
    bnd = S.elementwise_bound(A, W)
    assert np.all(np.abs(Yf - Yx) <= bnd)
    # the bound is not vacuous: errors reach a visible fraction of it
    assert np.max(np.abs(Yf - Yx) / bnd) > 1e-3


def test_rel_fro_error_definition():
    C = np.array([[3.0, 4.0]])
    assert S.rel_fro_error(C * (1 + 1e-3), C) == pytest.approx(1e-3)


def test_split3_close_to_exact():
    A = uniform(30, 200, 10)
    B = uniform(200, 12, 11)
    ex = A.astype(np.float64) @ B.astype(np.float64)
    em = S.split3_emulated(A, B)
    bound = 3 * S.U_FP16 ** 2 * (np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)))
    assert np.all(np.abs(em - ex) <= bound)


@pytest.mark.parametrize("pieces,tol", [(3, 2.0 ** -24), (2, 2.0 ** -16)])
def test_bf16_split_reconstruction(pieces, tol):
    A = uniform(50, 50, 12)
    ps = S.split_bf16(A, pieces)
    rec = sum(p * 2.0 ** (-8 * j) for j, p in enumerate(ps))
    a = A.astype(np.float64)
    assert np.all(np.abs(rec - a) <= tol * np.abs(a))


def test_range_flag():
    assert S.f16_range_ok(np.array([65519.0], dtype=np.float32))
    assert not S.f16_range_ok(np.array([65520.0], dtype=np.float32))
    assert not S.f16_range_ok(np.array([-1e6], dtype=np.float32))


def test_tf32_split_full_exponent_range():
    # SHGEMM-TF32 (Sec. 4.2): values far outside the FP16 range split and
    # reconstruct to within u^2 |a| (u = 2^-11, the TF32 unit roundoff), and
    # each piece has at most 11 significant bits
    rng = np.random.default_rng(21)
    e = rng.integers(-120, 120, size=4000)
    a = (rng.uniform(1.0, 2.0, size=4000) * np.exp2(e.astype(np.float64)) *
         rng.choice([-1.0, 1.0], size=4000)).astype(np.float32)
    hi, lo = S.split_tf32(a)
    a64 = a.astype(np.float64)
    assert np.all(np.isfinite(hi)) and np.all(np.isfinite(lo))
    rest = a64 - hi - lo * 2.0 ** -11
    assert np.all(np.abs(rest) <= (2.0 ** -11) ** 2 * np.abs(a64))
    for x in (hi, lo):
        nz = x != 0
        m, _ = np.frexp(x[nz])
        assert np.all(np.ldexp(m, 11) == np.rint(np.ldexp(m, 11)))   # <= 11 significant bits
    # the FP16 split cannot represent the large ones
    big = a[np.abs(a) >= 65520.0]
    assert big.size > 0 and not S.f16_range_ok(big)


def test_tf32_split_equals_fp16_split_where_both_are_exact():
    # TF32 and FP16 both carry 10 explicit mantissa bits: for a in [1, 2)
    # (hi and the scaled lo are FP16 normals) the two splits are the same
    rng = np.random.default_rng(22)
    a = rng.uniform(1.0, 2.0, size=5000).astype(np.float32)
    h16, l16 = S.split_f16(a)
    h32, l32 = S.split_tf32(a)
    keep = np.abs(l16) >= 2.0 ** -14          # lo an FP16 normal as well
    assert np.array_equal(h16, h32)
    assert np.array_equal(l16[keep], l32[keep])


def test_shgemm_tf32_emulated_integer_brute_force():
    rng = np.random.default_rng(23)
    A = rng.integers(-1000, 1000, size=(6, 9)).astype(np.float32)
    W = rng.integers(-30, 30, size=(9, 4)).astype(np.float16)
    ref = [[sum(int(A[i, l]) * int(W[l, j]) for l in range(9)) for j in range(4)] for i in range(6)]
    assert np.array_equal(S.shgemm_tf32_emulated(A, W), np.array(ref, dtype=np.float64))


def test_bf16_omega_matches_torch_cast_on_every_fp16_value():
    # RN_bf16 of each finite FP16 value: FP16 values are exact in float32, and
    # torch's float32 -> bfloat16 cast rounds to nearest even
    import torch
    from oracle.lowp import all_finite_values
    v = all_finite_values(FP16)
    got = S.bf16_omega(v.astype(np.float16))
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got, ref)


def test_shgemm_bf16_emulated_integer_brute_force():
    # integer A (|a| < 256: one BF16 piece, the others zero) and integer
    # Omega (|w| <= 256, exact in BF16) on a non-square case: the result is
    # the integer product, summed with Python integers
    rng = np.random.default_rng(5)
    A = rng.integers(-255, 256, size=(7, 11)).astype(np.float32)
    W = rng.integers(-256, 257, size=(11, 4)).astype(np.float16)
    ref = [[sum(int(A[i, l]) * int(W[l, j]) for l in range(11)) for j in range(4)] for i in range(7)]
    for pieces in (2, 3):
        assert np.array_equal(S.shgemm_bf16_emulated(A, W, pieces), np.array(ref, dtype=np.float64))


@pytest.mark.parametrize("pieces,u", [(3, 2.0 ** -24), (2, 2.0 ** -16)])
def test_shgemm_bf16_emulated_against_exact_product(pieces, u):
    # sum_j p_j 2^(-8j) reconstructs a within u |a| (the split's own pin), so
    # the emulated product is within u |A| |Omega_bf16| of A Omega_bf16; a
    # dropped piece or a missing 2^(-8j) scale is off by far more
    A = uniform(40, 300, 21)
    Om = omega_f16(300, 24, seed=22)
    W = S.bf16_omega(Om)
    ex = A.astype(np.float64) @ W
    em = S.shgemm_bf16_emulated(A, Om, pieces)
    bound = u * (1 + 2.0 ** -20) * (np.abs(A.astype(np.float64)) @ np.abs(W))
    assert np.all(np.abs(em - ex) <= bound)
    if pieces == 3:
        two = S.shgemm_bf16_emulated(A, Om, 2)
        assert np.max(np.abs(two - ex)) > 16 * np.max(np.abs(em - ex))
