"""Pins for oracle.rsvd (Algorithm 1, Eckart-Young, Eq. qqta-acc)."""
import numpy as np

from oracle import rsvd as R
from oracle.lowp import FP16, round_rn
from synth import omega_f16, planted_svd, sigma_exp, rsvd_planted


def _gram_schmidt(Y):
    """Classical Gram-Schmidt, float64, tiny well-conditioned inputs only."""
    m, k = Y.shape
    Q = np.zeros((m, k)); Rm = np.zeros((k, k))
    for j in range(k):
        v = Y[:, j].copy()
        for i in range(j):
            Rm[i, j] = Q[:, i] @ Y[:, j]
            v -= Rm[i, j] * Q[:, i]
        Rm[j, j] = np.sqrt(v @ v)
        Q[:, j] = v / Rm[j, j]
    return Q, Rm


def test_qr_pos_matches_gram_schmidt():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((9, 4))
    Q, Rr = R.qr_pos(Y)
    Qg, Rg = _gram_schmidt(Y)
    assert np.allclose(Q, Qg, atol=1e-12) and np.allclose(Rr, Rg, atol=1e-12)
    assert np.all(np.diag(Rr) > 0) and np.allclose(np.tril(Rr, -1), 0)


def test_exact_low_rank_recovery():
    sig = np.array([5.0, 3.0, 2.0, 1.0, 0.5, 0.25])
    A = planted_svd(120, 90, sig, seed=3)
    out = R.rsvd(A, omega_f16(90, 10, 4), p=6)
    assert out["r_k"] < 1e-6 and out["r_p"] < 1e-6       # limited by A's FP32 rounding
    assert np.allclose(out["S"], sig, rtol=1e-6)
    Q = out["Q"]
    assert np.linalg.norm(Q.T @ Q - np.eye(Q.shape[1])) < 1e-13


def test_full_width_sketch_gives_exact_svd():
    A = planted_svd(40, 30, sigma_exp(30, 4.0), seed=5)
    out = R.rsvd(A, omega_f16(30, 30, 6), p=12)
    s_ref = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    assert np.allclose(out["S"], s_ref[:12], rtol=1e-10)
    # residual equals the Eckart-Young value
    ey = R.eckart_young(s_ref, 12, np.linalg.norm(A.astype(np.float64)))
    assert abs(out["r_p"] - ey) < 1e-10


def test_eckart_young_lower_bound_and_factors():
    A, Om = rsvd_planted(256, 200, rate=8.0, seed_a=0, seed_omega=1, k=24)
    out = R.rsvd(A, Om, p=16)
    A64 = A.astype(np.float64)
    s_ref = np.linalg.svd(A64, compute_uv=False)
    ey = R.eckart_young(s_ref, 16, np.linalg.norm(A64))
    assert out["r_p"] >= ey * (1 - 1e-12)
    U, V = out["U"], out["V"]
    assert np.linalg.norm(U.T @ U - np.eye(16)) < 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(16)) < 1e-12
    # sigma estimates never exceed the true ones (Q^T A is a compression)
    assert np.all(out["S"] <= s_ref[:16] * (1 + 1e-12))


def test_halko_bound_in_expectation():
    p, s = 10, 6
    A = planted_svd(200, 150, sigma_exp(150, 6.0), seed=7)
    s_ref = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    errs = []
    for seed in range(10):
        out = R.rsvd(A, omega_f16(150, p + s, 100 + seed), p=p)
        errs.append(out["r_k"] * np.linalg.norm(A.astype(np.float64)))
    assert np.mean(errs) <= R.halko_bound(s_ref, p, s)
    assert np.mean(errs) >= R.eckart_young(s_ref, p + s)


def test_power_scheme_matches_closed_form():
    """With q = 1 the basis spans range((A A^T) A Omega) (Sec. 2.1)."""
    A = planted_svd(60, 50, sigma_exp(50, 2.0), seed=8)
    Om = omega_f16(50, 8, 9)
    out = R.rsvd(A, Om, p=5, q=1)
    A64 = A.astype(np.float64)
    Yc = A64 @ (A64.T @ (A64 @ Om.astype(np.float64)))
    Qc, _ = np.linalg.qr(Yc)
    Q = out["Q"]
    assert np.linalg.norm(Q @ Q.T - Qc @ Qc.T) < 1e-8
    out0 = R.rsvd(A, Om, p=5, q=0)
    assert out["r_k"] <= out0["r_k"]


def test_fp16_basis_reading_is_close():
    A = planted_svd(80, 70, sigma_exp(70, 4.0), seed=10)
    Om = omega_f16(70, 12, 11)
    a = R.rsvd(A, Om, p=6, q=1)
    b = R.rsvd(A, Om, p=6, q=1, fp16_basis=True)
    assert abs(a["r_p"] - b["r_p"]) < 0.01 * a["r_p"]
    assert np.allclose(a["S"], b["S"], rtol=1e-3)


def test_canonical_signs_hand_built():
    # column 0: largest |.| is -0.5 (row 1) -> flipped; column 1: largest is
    # +0.9 (row 0) -> kept; column 2: largest is -0.7 -> flipped.  V's
    # columns flip with U's, so U diag(s) V^T is unchanged.
    U = np.array([[0.1, 0.9, 0.2], [-0.5, 0.3, -0.7], [0.2, -0.1, 0.1]])
    V = np.array([[1.0, 2.0, 3.0], [-4.0, 5.0, -6.0]])
    Uc, Vc = R.canonical_signs(U, V)
    assert np.array_equal(Uc, U * np.array([-1.0, 1.0, -1.0]))
    assert np.array_equal(Vc, V * np.array([-1.0, 1.0, -1.0]))
    S = np.array([3.0, 2.0, 1.0])
    assert np.allclose((Uc * S) @ Vc.T, (U * S) @ V.T, rtol=0, atol=0)
    # already canonical columns are left alone; V may be omitted
    Uc2, none = R.canonical_signs(Uc)
    assert none is None and np.array_equal(Uc2, Uc)
    # a zero column keeps its sign (no NaN from sign(0))
    Z, _ = R.canonical_signs(np.zeros((3, 1)))
    assert np.array_equal(Z, np.zeros((3, 1)))
