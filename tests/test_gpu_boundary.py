"""GPU checks of the boundary pieces that state the problem as the paper
does (Algorithm 1: rank, oversampling, power iterations; Algorithm 2: mode
ranks and oversampling) and of the diagnostics report:

* shg_rsvd with a NULL Omega generates it from the seed as
  shg_gaussian_f16(seed, 0, n, k) does; the result matches the oracle run on
  those generated bytes (singular values within 1e-5, residual within 1 %).
* shg_rp_hosvd with NULL Omegas generates Omega_i as
  shg_gaussian_f16(seed, i * 2^32, rows_i, J_i) does; J_i = rank_i + s.
* The report: flags and status, the smallest Cholesky pivot ratio against
  the oracle's R_jj^2 / ||y_j||^2 of the basis (the first CholeskyQR pass
  dominates), the residual estimate against the oracle's estimate on the
  same probes and the same basis, and phase times that cover the call.
"""
import numpy as np
import pytest
import torch

from oracle import gaussian as OG
from oracle import hosvd as OH
from oracle import rsvd as OR
from oracle import shgemm as OS
from oracle import sketch as OSK
from synth import planted_svd, rsvd_planted, sigma_exp, tucker

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def shg():
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as m
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def generated(shg, seed, offset, rows, cols):
    """The library's Philox FP16 stream, fetched to the host (the bytes the
    call generates itself)."""
    buf = torch.empty(rows, (cols + 7) // 8 * 8, dtype=torch.float16, device="cuda")[:, :cols]
    return shg.shg_gaussian_f16(seed, offset, rows, cols, out=buf).cpu().numpy()


@pytest.mark.parametrize("variant", ["f16", "fp32", "bf16x3"])
def test_rsvd_null_omega_generated_from_seed(shg, variant):
    m, n, rank, s, seed = 800, 600, 24, 9, 31
    A = planted_svd(m, n, sigma_exp(min(m, n), 8.0), seed=3)
    U, S, V = shg.shg_rsvd(dev(A), None, rank, s, variant=variant, seed=seed)
    Om = generated(shg, seed, 0, n, rank + s)
    om = OS.bf16_omega(Om) if variant == "bf16x3" else Om
    ref = OR.rsvd(A, om, p=rank)
    S = S.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(S - ref["S"]) / ref["S"]) <= 1e-5
    A64 = A.astype(np.float64)
    U, V = U.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)
    r_p = np.linalg.norm(A64 - (U * S) @ V.T) / np.linalg.norm(A64)
    assert abs(r_p - ref["r_p"]) <= 0.01 * ref["r_p"]


@pytest.mark.parametrize("q", [0, 1])
def test_rsvd_report(shg, q):
    A, Om = rsvd_planted(1024, 1024, rate=8.0, seed_a=0, seed_omega=1, k=64)
    seed = 5
    buf = torch.zeros(1024, 64, dtype=torch.float16, device="cuda")
    buf[:] = dev(Om)
    U, S, V, Q, rep = shg.shg_rsvd(dev(A), buf, 32, 32, power_iters=q, want_q=True, seed=seed, report=True)
    assert rep["flags"] == 0 and rep["status"] == 0
    ref = OR.rsvd(A, Om, p=32, q=q, fp16_basis=True)
    # smallest pivot ratio: the first pass over Y = A Omega, R_jj^2 / ||y_j||^2
    # of its QR factor; ratios of later passes (near-orthonormal columns, or
    # the power scheme's better-conditioned bases) are larger
    A64 = A.astype(np.float64)
    Y = A64 @ Om.astype(np.float64)
    _, R = OR.qr_pos(Y)
    r_min = np.min(np.diag(R) ** 2 / np.sum(Y * Y, axis=0))
    if q == 0:
        assert abs(rep["min_pivot"] - r_min) <= 1e-2 * r_min, (rep["min_pivot"], r_min)
    else:
        assert 0.0 < rep["min_pivot"] <= r_min * 1.01
    # the residual estimate: the oracle's estimator on the same probes and
    # the returned basis Q (cancellation amplifies FP32 rounding by
    # ||A G|| / ||(I - Q Q^T) A G||)
    G = OG.gaussian_f16(seed, 1 << 62, 1024, 8)
    Q64 = Q.cpu().numpy().astype(np.float64)
    est_ref = OSK.residual_estimate(A, Q64, G, OG.alpha_Y(OG.FP16))
    AG = A64 @ G
    amp = np.linalg.norm(AG) / np.linalg.norm(AG - Q64 @ (Q64.T @ AG))
    tol = 64 * U32 * np.sqrt(64) * amp
    assert abs(rep["est_residual"] - est_ref) / est_ref <= tol, (rep["est_residual"], est_ref, tol)
    # ... and an unbiased estimate of the true residual r_k (8 probes: within a factor 2)
    assert 0.5 * ref["r_k"] <= rep["est_residual"] <= 2.0 * ref["r_k"]
    ph = rep["phase_ms"]
    assert all(v >= 0.0 for v in ph.values())
    for name in ("project", "orth", "B", "svd", "lift", "estimate"):
        assert ph[name] > 0.0, name
    if q == 0:
        assert ph["power"] < 0.05
    else:
        assert ph["power"] > ph["project"]
    # the report changes nothing in the results
    U2, S2, V2 = shg.shg_rsvd(dev(A), buf, 32, 32, power_iters=q, seed=seed)
    assert torch.allclose(S, S2, rtol=1e-6, atol=0)


def padded_f16(om):
    n, k = om.shape
    b = torch.zeros(n, (k + 7) // 8 * 8, dtype=torch.float16, device="cuda")
    b[:, :k] = dev(om)
    return b[:, :k]


def test_rp_hosvd_ranks_oversampling_and_null_omegas(shg):
    dims, ranks, s, seed = (64, 48, 40), (8, 6, 8), 4, 11
    J = [r + s for r in ranks]
    A, _, _ = tucker(dims, (8, 6, 8), seed=3, noise_std=1e-4)
    core, facs = shg.shg_rp_hosvd(dev(A), None, ranks, oversampling=s, seed=seed)
    assert tuple(core.shape) == tuple(J)
    oms = []
    for i in range(3):
        rows = int(np.prod([d for j, d in enumerate(dims) if j != i]))
        oms.append(generated(shg, seed, i << 32, rows, J[i]))
    ref = OH.rp_hosvd(A, oms)
    # the same call with the generated Omegas passed explicitly
    core2, facs2 = shg.shg_rp_hosvd(dev(A), [padded_f16(o) for o in oms], ranks, oversampling=s)
    for i in range(3):
        condW = np.linalg.cond(ref["W"][i])
        # both calls within the first-order QR perturbation of the oracle's
        # factor (the oversampled columns are noise-dominated, so cond(W_i)
        # amplifies the FP32 rounding of W_i, which differs run to run in
        # its last bits)
        for f in (facs[i], facs2[i]):
            F = f.cpu().numpy().astype(np.float64)
            assert F.shape == (dims[i], J[i])
            assert np.linalg.norm(F.T @ F - np.eye(J[i])) < 1e-5
            assert np.linalg.norm(F - ref["Q"][i]) <= 10 * condW * 1e-6 * np.sqrt(J[i])
    rec = OH.reconstruct(core.cpu().numpy(), [f.cpu().numpy() for f in facs])
    err = np.linalg.norm(A.astype(np.float64) - rec) / np.linalg.norm(A)
    assert abs(err - ref["err"]) <= 0.01 * ref["err"]
