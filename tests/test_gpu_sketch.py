"""GPU parity of the a-posteriori residual estimator (Theorems 1 and 3) and
of the learned-sketch loss and gradient against the FP64 oracle, plus the
autograd wiring, training and the Gaussian fallback.

Inputs come from the learned-sketch family of synth (rank-r signal with
rotated right factors plus relative noise).  The probes of the estimator
are the library's Philox FP16 Gaussians; the oracle regenerates the same
stream from (seed, offset) with its own Philox implementation.

Tolerances (u = 2^-24):
* estimate: the FP32 residual Z - Q (Q^T Z) cancels ||A G|| down to
  ||(I - QQ^T) A G||, so its relative error is about u * sqrt(k) *
  ||A G|| / ||(I - QQ^T) A G|| (times a safety factor of 64);
* loss: an absolute error of 64 u (FP32 projections, FP64 sums);
* gradient: the FP32 basis is accurate to about u cond(Y) and the projection
  (I - QQ^T) A A^T Q cancels ||A A^T Q|| down to its result, so the relative
  Frobenius error of dl/dOmega is bounded by 64 u cond(Y) ||A A^T Q|| / ||P||.
"""
import numpy as np
import pytest
import torch

from oracle import gaussian as OG
from oracle import sketch as OSK
from oracle.rsvd import qr_pos
from synth import sketch_basis, sketch_matrix

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


def family(m, n, r, seed, noise_rel=1e-2, basis_seed=100):
    V0 = sketch_basis(n, r, seed=basis_seed)
    sigma = 2.0 ** (-np.arange(1, r + 1) / 4.0)
    return sketch_matrix(V0, m, sigma, 0.2, noise_rel, seed)


def f16_omega(n, k, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, k)).astype(np.float32)


def dev_f16(om16):
    """FP16 n x k on the device with a leading dimension padded to 8."""
    n, k = om16.shape
    buf = torch.zeros(n, (k + 7) // 8 * 8, dtype=torch.float16, device="cuda")
    buf[:, :k] = torch.from_numpy(om16).cuda()
    return buf[:, :k]


@pytest.mark.parametrize("m,n,k,t", [(600, 520, 20, 16), (1030, 776, 40, 9)])
def test_residual_estimate_matches_oracle_same_probes(shg, m, n, k, t):
    A = family(m, n, 16, seed=1)
    Om = f16_omega(n, k, 2).astype(np.float16).astype(np.float64)
    Q, _ = qr_pos(A.astype(np.float64) @ Om)
    Q32 = Q.astype(np.float32)
    seed, offset = 77, 5
    out = shg.shg_residual_estimate(dev(A), dev(Q32), t=t, seed=seed, offset=offset).cpu().numpy()
    G = OG.gaussian_f16(seed, offset, n, t)
    alpha = OG.alpha_Y(OG.FP16)
    ref = OSK.residual_estimate(A, Q32.astype(np.float64), G, alpha)
    AG = A.astype(np.float64) @ G
    R = AG - Q32.astype(np.float64) @ (Q32.astype(np.float64).T @ AG)
    amp = np.linalg.norm(AG) / np.linalg.norm(R)
    tol = 64 * U32 * np.sqrt(k) * amp
    assert abs(out[0] - ref) / ref <= tol, (out[0], ref, tol)
    assert abs(out[2] - np.sum(A.astype(np.float64) ** 2)) / out[2] <= 64 * U32


def test_residual_estimate_is_unbiased(shg):
    # Theorems 1 and 3: E est^2 = ||(I - QQ^T) A||_F^2 / ||A||_F^2 for probes of
    # variance alpha; 96 probe sets of t = 16 give a relative standard error of
    # the mean of est^2 of a few per cent on this residual spectrum
    m, n, k, t = 800, 640, 24, 16
    A = family(m, n, 16, seed=3, noise_rel=5e-2)
    Om = f16_omega(n, k, 4).astype(np.float16).astype(np.float64)
    Q, _ = qr_pos(A.astype(np.float64) @ Om)
    A64 = A.astype(np.float64)
    true2 = np.sum((A64 - Q @ (Q.T @ A64)) ** 2) / np.sum(A64 ** 2)
    Ad, Qd = dev(A), dev(Q.astype(np.float32))
    est2 = [shg.shg_residual_estimate(Ad, Qd, t=t, seed=1000 + s)[0].item() ** 2 for s in range(96)]
    mean, sem = np.mean(est2), np.std(est2) / np.sqrt(len(est2))
    assert abs(mean - true2) <= 4 * sem + 1e-3 * true2, (mean, true2, sem)


@pytest.mark.parametrize("m,n,k", [(512, 384, 12), (700, 900, 33)])
def test_sketch_loss_and_gradient_match_oracle(shg, m, n, k):
    A = family(m, n, 8, seed=5)
    Om32 = f16_omega(n, k, 6)
    Om16 = Om32.astype(np.float16)
    Ad = dev(A)
    Y = shg.shgemm_project(Ad, dev_f16(Om16))
    loss, grad = shg.shg_sketch_loss_grad(Ad, Y)
    om = Om16.astype(np.float64)
    ref_loss = OSK.loss(A, om)
    assert abs(loss.item() - ref_loss) <= 64 * U32, (loss.item(), ref_loss)
    ref_grad = OSK.grad_omega(A, om)
    A64 = A.astype(np.float64)
    Yr = A64 @ om
    Q, R = qr_pos(Yr)
    M = A64 @ (A64.T @ Q)
    P = M - Q @ (Q.T @ M)
    tol = 64 * U32 * np.linalg.cond(Yr) * np.linalg.norm(M) / np.linalg.norm(P)
    err = np.linalg.norm(grad.cpu().numpy().astype(np.float64) - ref_grad) / np.linalg.norm(ref_grad)
    assert err <= tol, (err, tol)
    # loss only: the same value up to the summation order of the atomics
    loss2, g2 = shg.shg_sketch_loss_grad(Ad, Y, want_grad=False)
    assert g2 is None and abs(loss2.item() - loss.item()) <= 64 * U32


def test_sketchfn_autograd_and_training(shg):
    from paper_2304_04612_gb300.sketch import SketchFn
    m = n = 384
    k = r = 8          # no oversampling: a Gaussian sketch leaves a clear margin to learn
    train = [dev(family(m, n, r, seed=50 + i)) for i in range(12)]
    test = [dev(family(m, n, r, seed=500 + i)) for i in range(4)]
    torch.manual_seed(0)
    omega = torch.randn(n, k, device="cuda", requires_grad=True)
    # autograd delivers the library's gradient (equal up to the summation
    # order of the split-K atomics, amplified by the projection's cancellation)
    loss = SketchFn.apply(train[0], omega)
    loss.backward()
    om16 = torch.from_numpy(omega.detach().cpu().numpy().astype(np.float16))
    _, g_ref = shg.shg_sketch_loss_grad(train[0], shg.shgemm_project(train[0], dev_f16(om16.numpy())))
    assert torch.allclose(omega.grad, g_ref, rtol=1e-3, atol=1e-3 * g_ref.abs().max().item())
    omega.grad = None

    def test_loss():
        with torch.no_grad():
            return float(np.mean([SketchFn.apply(A, omega).item() for A in test]))

    before = test_loss()
    opt = torch.optim.Adam([omega], lr=0.05)
    for epoch in range(6):
        for A in train:
            opt.zero_grad()
            SketchFn.apply(A, omega).backward()
            opt.step()
    after = test_loss()
    assert after < 0.5 * before, (before, after)


def test_choose_sketch_falls_back_to_gaussian(shg):
    from paper_2304_04612_gb300.sketch import choose_sketch
    m = n = 512
    k, r = 12, 16
    A_h = family(m, n, r, seed=9)
    A = dev(A_h)
    V0 = sketch_basis(n, r, seed=100)
    # a poor "learned" sketch: directions orthogonal to the signal's basis
    rng = np.random.default_rng(11)
    X = rng.standard_normal((n, k))
    bad = (X - V0 @ (V0.T @ X)).astype(np.float32)
    om, est_l, est_g, used = choose_sketch(A, dev(bad), seed=4, probes=32)
    assert not used and est_l > est_g and om.dtype == torch.float16
    # the matrix's own leading right singular vectors beat a Gaussian sketch
    # with k < r columns
    V = np.linalg.svd(A_h.astype(np.float64), full_matrices=False)[2].T
    good = V[:, :k].astype(np.float32)
    om, est_l, est_g, used = choose_sketch(A, dev(good), seed=4, probes=32)
    assert used and est_l <= est_g
