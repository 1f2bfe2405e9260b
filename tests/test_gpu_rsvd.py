"""GPU parity of CholeskyQR2, the randomized SVD (Algorithm 1) and RP-HOSVD
(Algorithm 2) against the FP64 oracle fed the same FP32 A and FP16 Omega.

Tolerances: leading singular values within 1e-5 relative, the rank-p
residual ||A - U S V^T||_F / ||A||_F within 1% of the oracle's, Q^T Q = I
within 1e-5 (Frobenius), and the basis itself within the perturbation that
the FP32 rounding of Y allows (cond(Y) * relative error of Y).
"""
import numpy as np
import pytest
import torch

from oracle import rsvd as OR
from oracle import hosvd as OH  # noqa: F401  (rp_hosvd reference)
from oracle import shgemm as OS
from synth import rsvd_planted, omega_f16, planted_svd, sigma_exp, uniform, tucker, hosvd_omegas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shg():
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as m
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def padded_omega(Om):
    """n x k FP16 Omega stored with a leading dimension rounded up to a
    multiple of 8 (the 16-byte TMA row-stride rule); returns the n x k view."""
    n, k = Om.shape
    buf = torch.zeros(n, (k + 7) // 8 * 8, dtype=torch.float16, device="cuda")
    buf[:, :k] = dev(Om)
    return buf[:, :k]


def residual(A, U, S, V):
    A = A.astype(np.float64)
    return np.linalg.norm(A - (U.astype(np.float64) * S.astype(np.float64)) @ V.astype(np.float64).T) / np.linalg.norm(A)


def check_vectors(U, V, ref, eps=1e-5):
    """Singular vectors against the oracle's (same A, same Omega), up to the
    sign each pair (u_i, v_i) may take.  Wedin's theorem bounds the angle
    between a computed and an exact singular vector pair by ||E|| / delta_i,
    delta_i the distance of sigma_i to the other singular values of B; with
    the backward error ||E|| <= 1e-6 ||A|| of the FP32 pipeline (the level
    at which the singular values agree) and a factor 10 of slack, each
    vector is within eps sigma_1 / delta_i of the oracle's (eps = 1e-5).
    The pair's sign is unique: u_i and v_i must flip together."""
    S_all = np.asarray(ref["S_all"], dtype=np.float64)
    U = U.astype(np.float64)
    V = V.astype(np.float64)
    p = U.shape[1]
    for i in range(p):
        gaps = [S_all[i] - S_all[i + 1]] if i + 1 < len(S_all) else []
        if i > 0:
            gaps.append(S_all[i - 1] - S_all[i])
        tol = min(1.0, eps * S_all[0] / min(gaps))
        su = np.sign(U[:, i] @ ref["U"][:, i])
        sv = np.sign(V[:, i] @ ref["V"][:, i])
        assert su == sv, (i, su, sv)
        eu = np.linalg.norm(su * U[:, i] - ref["U"][:, i])
        ev = np.linalg.norm(sv * V[:, i] - ref["V"][:, i])
        assert eu <= tol and ev <= tol, (i, eu, ev, tol)


@pytest.mark.parametrize("m,k,cond", [(3000, 72, 1e4), (2000, 113, 1e4), (2000, 114, 1e4), (20000, 160, 1e6),
                                      (4096, 296, 2.6e5)])
def test_cholqr2_orthonormal_and_matches_householder(shg, m, k, cond):
    """CholeskyQR2 with the first Gram compensated and the second in working
    precision: orthonormal to a few FP32 units per entry whatever cond(X) up
    to ~1e6 (||Q^T Q - I||_F <= 2 k u, u = 2^-24: the second pass's Gram and
    triangular product each leave O(u) per entry), and the same factor as
    Householder QR to first order (cond u sqrt(k), shown where it is small).
    k = 113 is the largest one-CTA factorisation (its second pass in FP32),
    k = 114 the smallest on the panel path with R^-1 by 32 x 32 blocks (R
    padded to 128)."""
    rng = np.random.default_rng(0)
    U = np.linalg.qr(rng.standard_normal((m, k)))[0]
    V = np.linalg.qr(rng.standard_normal((k, k)))[0]
    X = ((U * np.logspace(0, -np.log10(cond), k)) @ V.T).astype(np.float32)
    Q = shg.shg_cholqr2(dev(X)).cpu().numpy().astype(np.float64)
    orth = np.linalg.norm(Q.T @ Q - np.eye(k))
    assert orth < 2 * k * 2.0 ** -24, orth
    if cond <= 1e4:
        Qr, _ = OR.qr_pos(X.astype(np.float64))
        assert np.linalg.norm(Q - Qr) < cond * 1e-6 * np.sqrt(k)


def test_cholqr2_not_spd_flag(shg):
    X = uniform(500, 16, seed=1)
    X[:, 5] = 0.0                               # exactly singular Gram matrix
    with pytest.raises(shg.ShgError) as ei:
        shg.shg_cholqr2(dev(X))
    assert ei.value.status == 3


@pytest.mark.parametrize("variant", ["f16", "fp32"])
def test_rsvd_planted_1024(shg, variant):
    """The randomized-SVD accuracy workload: 1024 x 1024, sigma_i = 2^(-i/8),
    rank 32, oversampling 32, q = 0."""
    A, Om = rsvd_planted(1024, 1024, rate=8.0, seed_a=0, seed_omega=1, k=64)
    U, S, V, Q = shg.shg_rsvd(dev(A), dev(Om), rank=32, oversampling=32, variant=variant, want_q=True)
    U, S, V, Q = (t.cpu().numpy() for t in (U, S, V, Q))
    ref = OR.rsvd(A, Om, p=32)
    rel_s = np.abs(S.astype(np.float64) - ref["S"]) / ref["S"]
    assert rel_s.max() <= 1e-5, rel_s.max()
    r_p = residual(A, U, S, V)
    assert abs(r_p - ref["r_p"]) <= 0.01 * ref["r_p"], (r_p, ref["r_p"])
    Q64 = Q.astype(np.float64)
    assert np.linalg.norm(Q64.T @ Q64 - np.eye(64)) <= 1e-5
    # basis: perturbation bound cond(Y) * ||dY|| / ||Y|| with ||dY||/||Y|| <= 1e-5
    condY = np.linalg.cond(ref["Y"])
    assert np.linalg.norm(Q64 - ref["Q"]) <= 10 * condY * 1e-6 * np.sqrt(64)
    # U, V orthonormal columns, and the oracle's vectors
    assert np.linalg.norm(U.T.astype(np.float64) @ U - np.eye(32)) < 1e-4
    assert np.linalg.norm(V.T.astype(np.float64) @ V - np.eye(32)) < 1e-4
    check_vectors(U, V, ref)


def test_rsvd_shgemm_no_worse_than_fp32(shg):
    A, Om = rsvd_planted(1024, 1024, rate=8.0, seed_a=0, seed_omega=1, k=64)
    ref = OR.rsvd(A, Om, p=32)
    out = {}
    for v in ("f16", "fp32"):
        U, S, V = shg.shg_rsvd(dev(A), dev(Om), rank=32, oversampling=32, variant=v)
        out[v] = residual(A, U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy())
    assert out["f16"] <= out["fp32"] * 1.01 + 1e-7
    assert abs(out["f16"] - ref["r_p"]) <= 0.01 * ref["r_p"]


@pytest.mark.parametrize("m,n,rank,s,q", [(700, 1200, 20, 12, 0), (1500, 600, 40, 16, 1), (512, 512, 16, 16, 2)])
def test_rsvd_shapes_and_power_scheme(shg, m, n, rank, s, q):
    A = planted_svd(m, n, sigma_exp(min(m, n), 16.0), seed=4)
    Om = omega_f16(n, rank + s, seed=5)
    U, S, V = shg.shg_rsvd(dev(A), dev(Om), rank=rank, oversampling=s, power_iters=q)
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    ref = OR.rsvd(A, Om, p=rank, q=q, fp16_basis=True)
    rel_s = np.abs(S.astype(np.float64) - ref["S"]) / ref["S"]
    assert rel_s.max() <= 1e-5, rel_s.max()
    r_p = residual(A, U, S, V)
    assert abs(r_p - ref["r_p"]) <= 0.01 * ref["r_p"]
    check_vectors(U, V, ref)


def test_rsvd_bf16_variant(shg):
    A, Om = rsvd_planted(1024, 1024, rate=8.0, seed_a=0, seed_omega=1, k=64)
    Wb = OS.bf16_omega(Om)
    from oracle.lowp import encode_bf16
    om_b = torch.from_numpy(encode_bf16(Wb).view(np.int16)).cuda().view(torch.bfloat16)
    U, S, V = shg.shg_rsvd(dev(A), om_b, rank=32, oversampling=32, variant="bf16x3")
    ref = OR.rsvd(A, Wb, p=32)
    rel_s = np.abs(S.cpu().numpy().astype(np.float64) - ref["S"]) / ref["S"]
    assert rel_s.max() <= 1e-5


def hosvd_checks(A, core, facs, ref, J):
    """Factors and core of Algorithm 2 against the oracle on the same Omegas:
    Q_i within the first-order QR perturbation 10 cond(W_i) 1e-6 sqrt(J_i)
    of the oracle's (W_i within 1e-6-level relative error), and the core
    within sum_i ||Q_i - Q_i^ref|| ||A|| / ||core|| + 1e-5 relative (each
    factor enters the core contraction once)."""
    core = core.cpu().numpy().astype(np.float64) if hasattr(core, "cpu") else core
    facs = [f.cpu().numpy().astype(np.float64) if hasattr(f, "cpu") else f for f in facs]
    dq = 0.0
    for i in range(3):
        F = facs[i]
        assert np.linalg.norm(F.T @ F - np.eye(J[i])) < 1e-5
        condW = np.linalg.cond(ref["W"][i])
        d = np.linalg.norm(F - ref["Q"][i])
        assert d <= 10 * condW * 1e-6 * np.sqrt(J[i]), (i, d, condW)
        dq += d
    nA = np.linalg.norm(A.astype(np.float64))
    tol = dq * nA / np.linalg.norm(ref["core"]) + 1e-5
    assert np.linalg.norm(core - ref["core"]) / np.linalg.norm(ref["core"]) <= tol
    return core, facs


def test_mode_projections_match_oracle(shg):
    """W_i = X_(i) Omega_i of every mode (mode 0 as a matrix, mode 1 through
    the 3-D tensor map, mode 2 transposed), element-wise against the exact
    product: relative Frobenius error <= 1e-5, no worse than 2x the FP32
    SIMT path (or the split's own representation error), every element
    within the Sec. 4.3 bound."""
    dims, J = (64, 48, 40), (12, 9, 16)
    A, _, _ = tucker(dims, (8, 8, 8), seed=3, noise_std=1e-4)
    oms = hosvd_omegas(dims, J, seed=4)
    X = dev(A)
    for i in range(3):
        om = torch.zeros(oms[i].shape[0], 16, dtype=torch.float16, device="cuda")
        om[:, :J[i]] = dev(oms[i])
        W = shg.shg_mode_project(X, om[:, :J[i]], i).cpu().numpy()
        Ws = shg.shg_mode_project(X, om[:, :J[i]], i, variant="fp32").cpu().numpy()
        Ai = OH.unfold(A, i)
        ref = OS.project_exact(Ai, oms[i])
        err, err_simt = OS.rel_fro_error(W, ref), OS.rel_fro_error(Ws, ref)
        err_repr = OS.rel_fro_error(OS.shgemm_emulated(Ai, oms[i]), ref)
        assert err <= 1e-5, (i, err)
        assert err <= max(2 * err_simt, 2 * err_repr), (i, err, err_simt, err_repr)
        assert err_simt <= 1e-5, (i, err_simt)
        bound = OS.elementwise_bound(Ai, oms[i]) + \
            OS.U_FP16 ** 2 * (np.abs(Ai.astype(np.float64)) @ np.abs(oms[i].astype(np.float64)))
        assert not (np.abs(W - ref) > bound * (1 + 1e-6) + 1e-30).any(), i


def test_rp_hosvd_small(shg):
    dims, J = (64, 48, 40), (12, 12, 12)
    A, _, _ = tucker(dims, (8, 8, 8), seed=3, noise_std=1e-4)
    oms = hosvd_omegas(dims, J, seed=4)
    ref = OH.rp_hosvd(A, oms)
    for variant in ("f16", "fp32"):
        # Omega stored with leading dimension 16 (the TMA row stride rule)
        om_d = []
        for o in oms:
            buf = torch.zeros(o.shape[0], 16, dtype=torch.float16, device="cuda")
            buf[:, :o.shape[1]] = dev(o)
            om_d.append(buf[:, :o.shape[1]])
        core, facs = shg.shg_rp_hosvd(dev(A), om_d, J, variant=variant)
        core, facs = hosvd_checks(A, core, facs, ref, J)
        # properties of the returned factorization, in plain float64 numpy
        rec = np.einsum("abc,ia,jb,kc->ijk", core, facs[0], facs[1], facs[2])
        err = np.linalg.norm(A.astype(np.float64) - rec) / np.linalg.norm(A)
        assert abs(err - ref["err"]) <= 0.01 * ref["err"], (variant, err, ref["err"])
        # the core is the projection of A on the returned factors (last step of Algorithm 2)
        proj = np.einsum("ijk,ia,jb,kc->abc", A.astype(np.float64), facs[0], facs[1], facs[2])
        assert np.linalg.norm(core - proj) / np.linalg.norm(proj) < 1e-5


def test_rsvd_large_k_grid_eigensolver(shg):
    """k = rank + s = 160 exceeds one SM's shared memory: the eigensolver runs
    as block Jacobi on the whole grid (cooperative launch).  Same tolerances
    as the other randomized-SVD cases (slower decay keeps sigma_128 / sigma_1
    = 2^-4)."""
    m, n, rank, s = 1200, 1000, 128, 32
    A = planted_svd(m, n, sigma_exp(min(m, n), 32.0), seed=8)
    Om = omega_f16(n, rank + s, seed=9)
    U, S, V = shg.shg_rsvd(dev(A), dev(Om), rank=rank, oversampling=s)
    U, S, V = (t.cpu().numpy() for t in (U, S, V))
    ref = OR.rsvd(A, Om, p=rank)
    rel_s = np.abs(S.astype(np.float64) - ref["S"]) / ref["S"]
    assert rel_s.max() <= 1e-5, rel_s.max()
    r_p = residual(A, U, S, V)
    assert abs(r_p - ref["r_p"]) <= 0.01 * ref["r_p"], (r_p, ref["r_p"])
    assert np.linalg.norm(U.T.astype(np.float64) @ U - np.eye(rank)) < 1e-4
    check_vectors(U, V, ref)


def test_rsvd_k_beyond_rotation_log(shg):
    """k = 296: the block solver on the whole grid, V transformed with A in
    every block round.  Same tolerances, on all 280 singular values and
    vectors."""
    m, n, rank, s = 900, 800, 280, 16
    A = planted_svd(m, n, sigma_exp(min(m, n), 64.0), seed=12)
    Om = omega_f16(n, rank + s, seed=13)
    U, S, V = shg.shg_rsvd(dev(A), dev(Om), rank=rank, oversampling=s)
    U, S, V = (t.cpu().numpy() for t in (U, S, V))
    ref = OR.rsvd(A, Om, p=rank)
    rel_s = np.abs(S.astype(np.float64) - ref["S"]) / ref["S"]
    assert rel_s.max() <= 1e-5, (int(rel_s.argmax()), rel_s.max())
    r_p = residual(A, U, S, V)
    assert abs(r_p - ref["r_p"]) <= 0.01 * ref["r_p"], (r_p, ref["r_p"])
    check_vectors(U, V, ref)


@pytest.mark.parametrize("m,n,rank,s,rate", [
    (700, 600, 17, 16, 8.0),      # k = 33: one-CTA Cholesky, one-CTA Jacobi
    (900, 700, 129, 16, 48.0),    # k = 145: panel Cholesky (k > 113), one-CTA Jacobi (k <= 158)
    (900, 800, 145, 16, 48.0),    # k = 161: block Jacobi on the grid (11 block pairs)
    (1000, 900, 281, 16, 96.0),   # k = 297: block Jacobi (19 block pairs)
    (1300, 1200, 561, 16, 192.0), # k = 577: block Jacobi (37 pairs), R^-1 by 32 x 32 blocks
])
def test_rsvd_odd_k(shg, m, n, rank, s, rate):
    """An odd k = rank + s reaches every k x k kernel (Cholesky, eigensolver,
    V, Rayleigh quotients, selection) padded to an even size (the one-CTA
    solver) or to a multiple of 16 (the block solver) with zero rows and
    columns; all p singular values and vectors against the oracle, the
    rank-p residual within 1 %."""
    A = planted_svd(m, n, sigma_exp(min(m, n), rate), seed=20 + rank)
    Om = omega_f16(n, rank + s, seed=21 + rank)
    U, S, V, Q = shg.shg_rsvd(dev(A), padded_omega(Om), rank=rank, oversampling=s, want_q=True)
    U, S, V, Q = (t.cpu().numpy() for t in (U, S, V, Q))
    ref = OR.rsvd(A, Om, p=rank)
    rel_s = np.abs(S.astype(np.float64) - ref["S"]) / ref["S"]
    assert rel_s.max() <= 1e-5, (int(rel_s.argmax()), rel_s.max())
    r_p = residual(A, U, S, V)
    assert abs(r_p - ref["r_p"]) <= 0.01 * ref["r_p"], (r_p, ref["r_p"])
    k = rank + s
    Q64 = Q.astype(np.float64)
    assert np.linalg.norm(Q64.T @ Q64 - np.eye(k)) <= 1e-5
    condY = np.linalg.cond(ref["Y"])
    assert np.linalg.norm(Q64 - ref["Q"]) <= 10 * condY * 1e-6 * np.sqrt(k)
    check_vectors(U, V, ref)
