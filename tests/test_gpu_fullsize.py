"""Parity at the full sizes of the five workloads, in the launch
configuration the benchmark times, on outputs the FP64 oracle computes one
by one:

* SHGEMM sweep (m = n = 4096, 8192, 16384; k = 64 .. 512; A U[-1,1] seed 2,
  Omega seed 1), autotuned launches: 64 sampled rows of Y per launch against
  the exact rows, relative Frobenius error <= 1e-5 and every element within
  the Sec. 4.3 bound.
* RP-HOSVD of the 512^3 Tucker tensor (J = 48): the oracle's Algorithm 2 on
  the same FP16 Omegas; reconstruction error within 1 % of the oracle's,
  orthonormal factors spanning the oracle's subspaces.
* Batched randomized SVD of the 256 uneven problems (s = 16, q = 1, one CUDA
  graph): three problems (the largest and two drawn at random) against the
  oracle on the same Philox Omegas.
* Learned sketch at 2048 x 2048, k = 96: loss and gradient against the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import shgemm as OS
from oracle import rsvd as OR
from oracle import hosvd as OH
from oracle import sketch as OSK
from oracle.rsvd import qr_pos
from synth import uniform, omega_f16, tucker, hosvd_omegas, batch_specs, sketch_basis, sketch_matrix

pytestmark = pytest.mark.gpu
KS = (64, 128, 256, 512)


@pytest.fixture(scope="module")
def shg():
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as m
    return m


@pytest.mark.parametrize("mn", [4096, 8192, 16384])
def test_shgemm_sweep_sampled_rows(shg, mn):
    A = uniform(mn, mn, seed=2)
    Om = omega_f16(mn, max(KS), seed=1)
    Ad = torch.from_numpy(A).cuda()
    Od = torch.from_numpy(Om).cuda()
    rows = np.sort(np.random.default_rng(mn).choice(mn, size=64, replace=False))
    for k in KS:
        Y = torch.empty(mn, k, device="cuda")
        shg.shg_autotune_project(Ad, Od[:, :k], reps=1, out=Y)
        shg.shgemm_project(Ad, Od[:, :k], out=Y)
        Ys = Y[torch.from_numpy(rows).cuda()].cpu().numpy()
        ref = OS.project_exact(A[rows], Om[:, :k])
        err = OS.rel_fro_error(Ys, ref)
        assert err <= 1e-5, (mn, k, err)
        bound = OS.elementwise_bound(A[rows], Om[:, :k]) + \
            OS.U_FP16 ** 2 * (np.abs(A[rows].astype(np.float64)) @ np.abs(Om[:, :k].astype(np.float64)))
        assert not (np.abs(Ys - ref) > bound * (1 + 1e-6) + 1e-30).any(), (mn, k)
    shg.shg_autotune_clear()


def test_rp_hosvd_512_cubed(shg):
    dims, J = (512, 512, 512), (48, 48, 48)
    A, _, _ = tucker(dims, (32, 32, 32), seed=3, noise_std=1e-4)
    oms = hosvd_omegas(dims, J, seed=3)
    ref = OH.rp_hosvd(A, oms)
    X = torch.from_numpy(A).cuda()
    core, facs = shg.shg_rp_hosvd(X, [torch.from_numpy(o).cuda() for o in oms], J)
    Fs = [f.double() for f in facs]
    rec = torch.einsum("abc,ia,jb,kc->ijk", core.double(), Fs[0], Fs[1], Fs[2])
    err = float(torch.linalg.norm(X.double() - rec) / torch.linalg.norm(X.double()))
    assert abs(err - ref["err"]) <= 0.01 * ref["err"], (err, ref["err"])
    dq = 0.0
    for i in range(3):
        F = Fs[i].cpu().numpy()
        assert np.linalg.norm(F.T @ F - np.eye(J[i])) < 1e-5
        # factors within the first-order QR perturbation of the oracle's
        condW = np.linalg.cond(ref["W"][i])
        d = np.linalg.norm(F - ref["Q"][i])
        assert d <= 10 * condW * 1e-6 * np.sqrt(J[i]), (i, d, condW)
        dq += d
    # core within the factors' perturbation (each enters the contraction once)
    c = core.double().cpu().numpy()
    tol = dq * np.linalg.norm(A.astype(np.float64)) / np.linalg.norm(ref["core"]) + 1e-5
    assert np.linalg.norm(c - ref["core"]) / np.linalg.norm(ref["core"]) <= tol
    # every mode projection W_i = X_(i) Omega_i element-wise against the exact
    # product on 64 sampled rows (relative Frobenius <= 1e-5, Sec. 4.3 bound)
    rows = np.sort(np.random.default_rng(9).choice(512, size=64, replace=False))
    for i in range(3):
        W = shg.shg_mode_project(X, torch.from_numpy(oms[i]).cuda(), i).cpu().numpy()[rows]
        Ai = OH.unfold(A, i)[rows]
        refW = OS.project_exact(Ai, oms[i])
        assert OS.rel_fro_error(W, refW) <= 1e-5, i
        bound = OS.elementwise_bound(Ai, oms[i]) + \
            OS.U_FP16 ** 2 * (np.abs(Ai.astype(np.float64)) @ np.abs(oms[i].astype(np.float64)))
        assert not (np.abs(W - refW) > bound * (1 + 1e-6) + 1e-30).any(), i


def test_batched_256_sampled_problems(shg):
    specs = batch_specs(256, seed=4)
    g = torch.Generator(device="cuda").manual_seed(4)
    As, ranks = [], []
    for sp in specs:
        m, n = sp["m"], sp["n"]
        r = min(m, n, 256)
        sig = torch.pow(2.0, -torch.arange(1, r + 1, device="cuda", dtype=torch.float32) / sp["rate"])
        q1 = torch.linalg.qr(torch.randn(m, r, device="cuda", generator=g))[0]
        q2 = torch.linalg.qr(torch.randn(n, r, device="cuda", generator=g))[0]
        buf = torch.zeros(m, (n + 3) // 4 * 4, device="cuda")
        buf[:, :n] = (q1 * sig) @ q2.T
        As.append(buf[:, :n])
        ranks.append(sp["rank"])
    s, q, seed = 16, 1, 4
    Us, Ss, Vs = shg.shg_rsvd_batched(As, ranks, s, q, omegas=None, seed=seed, use_graph=True)
    big = int(np.argmax([A.shape[0] * A.shape[1] for A in As]))
    # the worst-conditioned sketches: sigma_1 / sigma_k = 2^(k / rate) is
    # largest for k = 144 at the fastest decay (about 2^18), where the
    # compensated-FP32 Gram matrix of CholeskyQR is under the most strain
    cond_log2 = [(r + s) / sp["rate"] for r, sp in zip(ranks, specs)]
    worst = [int(i) for i in np.argsort(cond_log2)[::-1][:2]]
    pick = [big] + worst + list(np.random.default_rng(5).choice(256, size=2, replace=False))
    for i in pick:
        A = As[i].cpu().numpy()
        n, k = A.shape[1], ranks[i] + s
        om = shg.shg_gaussian_f16(seed, int(i) << 32, n, k,
                                  out=torch.empty(n, (k + 7) // 8 * 8, dtype=torch.float16, device="cuda")[:, :k])
        ref = OR.rsvd(A, om.cpu().numpy(), p=ranks[i], q=q, fp16_basis=True)
        S = Ss[i].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(S - ref["S"]) / ref["S"]) <= 1e-5, i
        A64 = A.astype(np.float64)
        U, V = Us[i].cpu().numpy().astype(np.float64), Vs[i].cpu().numpy().astype(np.float64)
        r_p = np.linalg.norm(A64 - (U * S) @ V.T) / np.linalg.norm(A64)
        assert abs(r_p - ref["r_p"]) <= 0.01 * ref["r_p"], (i, r_p, ref["r_p"])


def test_learned_sketch_2048(shg):
    n, k, r = 2048, 96, 64
    V0 = sketch_basis(n, r, seed=100)
    A = sketch_matrix(V0, n, 2.0 ** (-np.arange(1, r + 1) / 8.0), 0.2, 1e-3, seed=5)
    Om16 = np.random.default_rng(6).standard_normal((n, k)).astype(np.float16)
    Ad = torch.from_numpy(A).cuda()
    Od = torch.from_numpy(Om16).cuda()
    Y = shg.shgemm_project(Ad, Od)
    loss, grad = shg.shg_sketch_loss_grad(Ad, Y)
    om = Om16.astype(np.float64)
    U32 = 2.0 ** -24
    assert abs(loss.item() - OSK.loss(A, om)) <= 64 * U32
    ref_grad = OSK.grad_omega(A, om)
    A64 = A.astype(np.float64)
    Yr = A64 @ om
    Q, _ = qr_pos(Yr)
    M = A64 @ (A64.T @ Q)
    P = M - Q @ (Q.T @ M)
    tol = 64 * U32 * np.linalg.cond(Yr) * np.linalg.norm(M) / np.linalg.norm(P)
    err = np.linalg.norm(grad.cpu().numpy().astype(np.float64) - ref_grad) / np.linalg.norm(ref_grad)
    assert err <= tol, (err, tol)
