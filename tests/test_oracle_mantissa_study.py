"""The low-precision Gaussian study (oracle/mantissa_study.py): the random
projection is about as accurate with G rounded to short mantissas as with
FP32 G, for both input types (the paper's conclusion of the experiment).
n = 512 instead of 4096 keeps the test in seconds; the pins are the
format-independence (16-bit and TF32-like formats within 1 %, 8-bit and
1-2-bit mantissas within 10 % of the FP32 G's error over three draws) and a
sanity check of the matrices' construction."""
import numpy as np
import pytest

from oracle import mantissa_study as MS


@pytest.mark.parametrize("kind", ["type1", "type2"])
def test_error_independent_of_mantissa_length(kind):
    n, r, k = 512, 20, 30
    A = MS.type1(n, r, 1e-4, seed=1) if kind == "type1" else MS.type2(n, r, 3.0, 1e6, seed=2)
    for seed in range(3):
        res = MS.study(A, k, seed=10 + seed)
        base = res["e8m23"]
        for f in ("e8m10", "fp16", "bf16"):
            assert abs(res[f] / base - 1) < 0.01, (kind, seed, f, res[f] / base)
        for f in ("fp8_e4m3", "fp8_e5m2", "e8m2", "e8m1"):
            assert abs(res[f] / base - 1) < 0.10, (kind, seed, f, res[f] / base)


def test_matrix_construction():
    n, r = 256, 20
    A2 = MS.type2(n, r, 3.0, 1e6, seed=2).astype(np.float64)
    s = np.linalg.svd(A2, compute_uv=False)
    # phi = 1e6 on r directions, then 2^-3; further down the FP32 rounding of
    # the entries (about 1e6 * 2^-24 each) is larger than the planted values
    assert np.allclose(s[:r], 1e6, rtol=1e-6) and abs(s[r] - 0.125) < 0.005 and s[r + 1] < 0.06
    A1 = MS.type1(n, r, 1e-4, seed=1).astype(np.float64)
    assert np.allclose(A1, A1.T, atol=1e-6) and np.linalg.eigvalsh(A1).min() > -1e-6
    # r eigenvalues near 1, the rest at the noise level xi * (eigenvalues of G G^T / n) <= 4e-4
    ev = np.sort(np.linalg.eigvalsh(A1))[::-1]
    assert np.all(ev[:r] > 0.99) and ev[r] < 1e-3


def test_projection_error_eckart_young():
    # with G the top-k right singular vectors of A (numpy's SVD), range(A G)
    # is the top-k left singular subspace and the error is the tail of the
    # singular values; with G spanning all of range(A^T) the error vanishes
    # (an integer product: A is exactly rank 15 in FP32 as well)
    rng = np.random.default_rng(4)
    A = (rng.integers(-3, 4, (60, 15)) @ rng.integers(-3, 4, (15, 50))).astype(np.float32)
    A64 = A.astype(np.float64)
    _, s, Vt = np.linalg.svd(A64)
    for k in (1, 5, 12):
        assert s[k] > 1e-3 * s[0]
        e = MS.projection_error(A, Vt[:k].T)
        assert np.isclose(e, np.sqrt(np.sum(s[k:] ** 2)), rtol=1e-10)
    G = rng.standard_normal((50, 20))
    assert MS.projection_error(A, G) < 1e-10 * np.linalg.norm(A64)
