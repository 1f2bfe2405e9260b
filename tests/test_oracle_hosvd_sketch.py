"""Pins for oracle.hosvd (Algorithm 2) and oracle.sketch (loss, gradient, estimator)."""
import numpy as np

from oracle import hosvd as H
from oracle import sketch as K
from oracle import rsvd as R
from oracle.gaussian import alpha_Y
from oracle.lowp import FP16
from synth import tucker, hosvd_omegas, planted_svd, sigma_exp, omega_f16


def test_unfold_index_convention():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((3, 4, 5))
    U1 = H.unfold(A, 1)
    for i1 in range(3):
        for i2 in range(4):
            for i3 in range(5):
                assert U1[i2, i1 * 5 + i3] == A[i1, i2, i3]
    U2 = H.unfold(A, 2)
    assert U2[4, 2 * 4 + 3] == A[2, 3, 4]


def test_mode_products_brute_force():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((3, 4, 2))
    Q = rng.standard_normal((4, 3))
    T = H.mode_product_T(A, Q, 1)
    for a in range(3):
        for j in range(3):
            for c in range(2):
                assert np.isclose(T[a, j, c], sum(A[a, b, c] * Q[b, j] for b in range(4)))
    B = H.mode_product(T, Q, 1)
    for a in range(3):
        for b in range(4):
            for c in range(2):
                assert np.isclose(B[a, b, c], sum(T[a, j, c] * Q[b, j] for j in range(3)))


def test_exact_tucker_recovery_without_noise():
    A, core, facs = tucker((20, 18, 16), (4, 3, 5), seed=3, noise_std=0.0)
    om = hosvd_omegas(A.shape, (6, 5, 7), seed=4)
    out = H.rp_hosvd(A, om)
    assert out["err"] < 1e-6                      # A is stored in FP32
    for Q in out["Q"]:
        assert np.linalg.norm(Q.T @ Q - np.eye(Q.shape[1])) < 1e-12
    rec = H.reconstruct(out["core"], out["Q"])
    assert np.linalg.norm(rec - A.astype(np.float64)) / np.linalg.norm(A) < 1e-6


def test_noise_floor_small_noise():
    A, _, _ = tucker((24, 24, 24), (4, 4, 4), seed=5, noise_std=1e-4)
    out = H.rp_hosvd(A, hosvd_omegas(A.shape, (8, 8, 8), seed=6))
    noise_rel = 1e-4 * np.sqrt(A.size) / np.linalg.norm(A)
    # the error is the noise outside the captured subspaces plus the signal
    # leaked by the sketch noise (||N Omega|| / sigma_min(S Omega) ~ 1e-2 here):
    # both are of the order of the noise level
    assert 0.5 * noise_rel < out["err"] < 3.0 * noise_rel


def test_nested_sketches_error_non_increasing():
    """Prefixes of one Omega span nested subspaces, so the orthogonal Tucker
    projection error cannot grow with J."""
    A, _, _ = tucker((16, 16, 16), (4, 4, 4), seed=7, noise_std=1e-2)
    full = hosvd_omegas(A.shape, (16, 16, 16), seed=8)
    errs = [H.rp_hosvd(A, [om[:, :J] for om in full])["err"] for J in (4, 6, 8, 12, 16)]
    assert all(b <= a + 1e-12 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-12


def test_sketch_gradient_finite_differences():
    A = planted_svd(30, 20, sigma_exp(20, 3.0), seed=7).astype(np.float64)
    Om = omega_f16(20, 5, 8).astype(np.float64)
    g = K.grad_omega(A, Om)
    idx = [(0, 0), (3, 2), (19, 4), (10, 1)]
    fd = K.grad_omega_fd(A, Om, idx, h=1e-6)
    assert np.allclose([g[i, j] for i, j in idx], fd, rtol=1e-5, atol=1e-9)


def test_sketch_loss_matches_range_finder_residual():
    A = planted_svd(50, 40, sigma_exp(40, 4.0), seed=9)
    Om = omega_f16(40, 8, 10)
    l = K.loss(A.astype(np.float64), Om.astype(np.float64))
    r = R.rsvd(A, Om, p=4)["r_k"]
    assert np.isclose(l, r * r, rtol=1e-10)


def test_residual_estimator_unbiased():
    A = planted_svd(60, 50, sigma_exp(50, 5.0), seed=11).astype(np.float64)
    Q, _ = R.qr_pos(A @ omega_f16(50, 6, 12).astype(np.float64))
    true = np.linalg.norm(A - Q @ (Q.T @ A)) / np.linalg.norm(A)
    al = alpha_Y(FP16)
    ests = [K.residual_estimate(A, Q, omega_f16(50, 16, 100 + s).astype(np.float64), al) ** 2
            for s in range(200)]
    assert abs(np.mean(ests) / true ** 2 - 1.0) < 0.05


def test_sketch_gradient_in_y_finite_differences():
    # dl/dY for a generic Y (not in the range of A, m > n so that A^T has a
    # null space): central differences of l(Y) = 1 - ||Q^T A||^2 / ||A||^2,
    # Q from the QR of Y, written out here.  grad_omega's own pin cannot see
    # a slip in the part of dl/dY that A^T maps to zero
    rng = np.random.default_rng(13)
    A = planted_svd(25, 12, sigma_exp(12, 2.0), seed=14).astype(np.float64)
    Y = rng.standard_normal((25, 4))
    nA2 = np.sum(A * A)

    def l(Yv):
        Q, _ = np.linalg.qr(Yv)
        return 1.0 - np.sum((Q.T @ A) ** 2) / nA2

    g = K.grad_Y(A, Y)
    h = 1e-6
    for i, j in [(0, 0), (24, 3), (7, 1), (13, 2)]:
        Yp = Y.copy(); Yp[i, j] += h
        Ym = Y.copy(); Ym[i, j] -= h
        assert np.isclose(g[i, j], (l(Yp) - l(Ym)) / (2 * h), rtol=1e-5, atol=1e-9)
