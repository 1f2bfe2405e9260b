"""The seeded input generators produce what their recipes state (shapes,
orthonormality, spectra, ranges, rounding), so that every workload that
the tests and the benchmark describe is the one they get."""
import numpy as np

from synth import (batch_matrix, batch_specs, haar, hosvd_omegas, omega_f16, planted_svd, rsvd_planted,
                   sigma_exp, sketch_basis, sketch_matrix, tucker, uniform)


def test_haar_columns_orthonormal():
    Q = haar(200, 30, np.random.default_rng(0))
    assert Q.shape == (200, 30)
    assert np.abs(Q.T @ Q - np.eye(30)).max() < 1e-12


def test_omega_is_fp32_gaussian_rounded_to_fp16():
    Om = omega_f16(64, 8, seed=3)
    g = np.random.default_rng(3).standard_normal((64, 8), dtype=np.float32)
    assert Om.dtype == np.float16
    assert np.array_equal(Om, g.astype(np.float16))


def test_planted_spectrum_and_rsvd_workload():
    sig = sigma_exp(40, 8.0)
    assert np.allclose(sig[:3], 2.0 ** (-np.arange(1, 4) / 8.0))
    A = planted_svd(120, 90, sig, seed=1)
    assert A.dtype == np.float32 and A.shape == (120, 90)
    s = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    assert np.allclose(s[:40], sig, rtol=1e-5, atol=1e-7)
    assert s[40:].max() < 1e-6
    A, Om = rsvd_planted(256, 200, rate=8.0, seed_a=0, seed_omega=1, k=24)
    assert A.shape == (256, 200) and Om.shape == (200, 24)


def test_uniform_range():
    U = uniform(100, 50, seed=2)
    assert U.dtype == np.float32 and U.min() >= -1.0 and U.max() < 1.0


def test_tucker_multilinear_rank_without_noise():
    A, core, facs = tucker((20, 16, 12), (4, 3, 2), seed=5, noise_std=0.0)
    for mode, r in enumerate((4, 3, 2)):
        unf = np.moveaxis(A.astype(np.float64), mode, 0).reshape(A.shape[mode], -1)
        s = np.linalg.svd(unf, compute_uv=False)
        assert s[r] < 1e-5 * s[0] and s[r - 1] > 1e-3 * s[0]
    assert np.linalg.norm(core) > 0 and all(f.shape[1] == r for f, r in zip(facs, (4, 3, 2)))


def test_hosvd_omegas_shapes():
    oms = hosvd_omegas((6, 5, 4), (3, 2, 2), seed=1)
    assert [o.shape for o in oms] == [(20, 3), (24, 2), (30, 2)]
    assert all(o.dtype == np.float16 for o in oms)


def test_batch_specs_ranges_and_clipping():
    sp = batch_specs(256, seed=4)
    m = np.array([p["m"] for p in sp]); n = np.array([p["n"] for p in sp])
    rank = np.array([p["rank"] for p in sp]); rate = np.array([p["rate"] for p in sp])
    assert m.min() >= 256 and m.max() <= 4096 and n.min() >= 256 and n.max() <= 2048
    assert rate.min() >= 8 and rate.max() <= 64
    assert set(rank.tolist()) <= {16, 32, 64, 128}
    assert np.all(rank + 16 <= np.minimum(m, n))
    small = batch_specs(50, seed=1, m_range=(20, 40), n_range=(20, 40))
    assert all(p["rank"] + 16 <= min(p["m"], p["n"]) for p in small)
    assert any(p["rank"] < 16 for p in small)                          # clipped
    A = batch_matrix(dict(m=60, n=40, rate=8.0, rank=8, seed=3))
    s = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    assert np.allclose(s, sigma_exp(40, 8.0), rtol=1e-5, atol=1e-7)


def test_sketch_family_angles_and_noise():
    n, r, m = 120, 6, 80
    V0 = sketch_basis(n, r, seed=100)
    sig = 2.0 ** (-np.arange(1, r + 1) / 4.0)
    A = sketch_matrix(V0, m, sig, theta_max=0.2, noise_rel=0.0, seed=7).astype(np.float64)
    # noise-free: rank r, right singular subspace within 0.2 rad of span(V0)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    assert s[r] < 1e-5 * s[0]
    cosines = np.linalg.svd(V0.T @ Vt[:r].T, compute_uv=False)
    assert cosines.min() >= np.cos(0.2) - 1e-5
    B = sketch_matrix(V0, m, sig, theta_max=0.2, noise_rel=1e-2, seed=7).astype(np.float64)
    assert abs(np.linalg.norm(B - A) / np.linalg.norm(A) - 1e-2) < 1e-4
