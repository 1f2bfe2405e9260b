"""SHGEMM-TF32 (Sec. 4.2: A split into TF32 hi and 2^11-scaled TF32 lo, the
FP16 Omega widened exactly to TF32) and the automatic fallback to it when
SHGEMM-FP16's range check trips (|a| >= 65520, the Cauchy matrices of
Sec. 5.1), against the FP64 oracle on the same FP32 A and FP16 Omega.

Tolerances: as for SHGEMM-FP16 (TF32 and FP16 have the same unit roundoff
2^-11): relative Frobenius error <= 1e-5, no worse than 2x the FP32 SIMT
path or the split's own representation error, every element within
(1/8) n u |A||Omega| + u_tf32^2 |A||Omega| (transposed products run in FP32
SIMT: within n u |A||Omega|, the sequential-sum bound)."""
import numpy as np
import pytest
import torch

from oracle import hosvd as OH
from oracle import rsvd as OR
from oracle import shgemm as OS
from synth import cauchy_family, omega_f16, planted_svd, sigma_exp, tucker, hosvd_omegas, uniform

pytestmark = pytest.mark.gpu
SHAPES = [(300, 1000, 64), (129, 67, 1), (256, 512, 200), (1000, 300, 256), (64, 4096, 48), (513, 2048, 96),
          (77, 1536, 144)]


@pytest.fixture(scope="module")
def shg():
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as m
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def padded_f32(A):
    r, c = A.shape
    buf = torch.zeros(r, (c + 3) // 4 * 4, dtype=torch.float32, device="cuda")
    buf[:, :c] = dev(A)
    return buf[:, :c]


def padded_f16(Om):
    n, k = Om.shape
    buf = torch.zeros(n, (k + 7) // 8 * 8, dtype=torch.float16, device="cuda")
    buf[:, :k] = dev(Om)
    return buf[:, :k]


def check_product(Y, A_op, Om, Ys, transposed):
    ref = OS.project_exact(A_op, Om)
    err, err_simt = OS.rel_fro_error(Y, ref), OS.rel_fro_error(Ys, ref)
    err_repr = OS.rel_fro_error(OS.shgemm_tf32_emulated(A_op, Om), ref)
    assert err <= 1e-5, (err, err_simt)
    assert err <= max(2.0 * err_simt, 2.0 * err_repr), (err, err_simt, err_repr)
    absprod = np.abs(A_op.astype(np.float64)) @ np.abs(Om.astype(np.float64))
    n = A_op.shape[1]
    if transposed:
        bound = n * OS.U_FP32 * absprod
    else:
        bound = OS.elementwise_bound(A_op, Om) * (1 if n >= 8 else 8.0 / n) + OS.U_FP16 ** 2 * absprod
    viol = np.abs(Y - ref) > bound * (1 + 1e-6) + 1e-30
    assert not viol.any(), f"{viol.sum()} elements exceed the bound"


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("trans", [False, True])
def test_shgemm_tf32_parity(shg, m, n, k, trans):
    A = uniform(n, m, seed=2) if trans else uniform(m, n, seed=2)
    Om = omega_f16(n, k, seed=1)
    A_op = A.T.copy() if trans else A
    Y = shg.shgemm_project(padded_f32(A), padded_f16(Om), "tf32", trans_a=trans).cpu().numpy()
    Ys = shg.shgemm_project(padded_f32(A), padded_f16(Om), "fp32", trans_a=trans).cpu().numpy()
    check_product(Y, A_op, Om, Ys, trans)


@pytest.mark.parametrize("scale_log2", [-100, -40, 40, 100])
def test_shgemm_tf32_full_exponent_range(shg, scale_log2):
    """A scaled far outside the FP16 range (both ways): the TF32 split keeps
    FP32's exponent range, so the relative accuracy does not change.  (Scales
    whose products fall below FP32's smallest normal number, 2^-126, lose
    accuracy: the tensor core does not keep FP32 subnormals.)"""
    m, n, k = 300, 700, 96
    A = (uniform(m, n, seed=5).astype(np.float64) * 2.0 ** scale_log2).astype(np.float32)
    Om = omega_f16(n, k, seed=6)
    Y = shg.shgemm_project(padded_f32(A), padded_f16(Om), "tf32").cpu().numpy()
    ref = OS.project_exact(A, Om)
    assert OS.rel_fro_error(Y, ref) <= 1e-5
    assert OS.rel_fro_error(OS.shgemm_tf32_emulated(A, Om), ref) <= 1e-6


def test_auto_falls_back_on_cauchy_matrix(shg):
    """The Cauchy stand-in (entries ~1e14) overflows the FP16 split: the
    FP16 variant reports SHG_ERR_RANGE; the automatic variant redoes the
    product with SHGEMM-TF32, leaves the flags word as it was and matches the
    exact product; on in-range data it is the FP16 result."""
    A = cauchy_family(512, seed=7)
    assert np.abs(A).max() > 65520
    Om = omega_f16(512, 64, seed=8)
    Ad, Od = padded_f32(A), padded_f16(Om)
    with pytest.raises(shg.ShgError) as ei:
        shg.shgemm_project(Ad, Od, "f16")
    assert ei.value.status == 2
    fl = shg.new_flags()
    Y = shg.shgemm_project(Ad, Od, "auto", flags=fl).cpu().numpy()
    assert int(fl.item()) == 0
    ref = OS.project_exact(A, Om)
    assert OS.rel_fro_error(Y, ref) <= 1e-5
    Yt = shg.shgemm_project(Ad, Od, "tf32").cpu().numpy()
    assert OS.rel_fro_error(Y, Yt) <= 1e-6
    B = uniform(400, 512, seed=9)
    Yb = shg.shgemm_project(padded_f32(B), Od, "auto").cpu().numpy()
    Yf = shg.shgemm_project(padded_f32(B), Od, "f16").cpu().numpy()
    assert OS.rel_fro_error(Yb, OS.project_exact(B, Om)) <= 1e-5
    assert OS.rel_fro_error(Yb, Yf) <= 1e-6


@pytest.mark.parametrize("q", [0, 1])
def test_rsvd_auto_and_tf32_full_range(shg, q):
    """Randomized SVD of a matrix whose entries exceed the FP16 range (the
    planted-spectrum matrix scaled by 2^24): SHG_SPLIT_F16 fails with
    SHG_ERR_RANGE, SHG_SPLIT_TF32 and SHG_SPLIT_AUTO match the oracle
    (singular values within 1e-5, residual within 1 %)."""
    m, n, rank, s = 700, 600, 24, 16
    A = (planted_svd(m, n, sigma_exp(min(m, n), 8.0), seed=3).astype(np.float64) * 2.0 ** 24).astype(np.float32)
    assert np.abs(A).max() > 65520
    Om = omega_f16(n, rank + s, seed=4)
    Ad, Od = padded_f32(A), padded_f16(Om)
    fl = shg.new_flags()
    shg.shg_rsvd(Ad, Od, rank, s, power_iters=q, variant="f16", flags=fl, check=False)
    assert int(fl.item()) & shg.FLAG_RANGE     # (the infinite Y also breaks CholeskyQR: NOT_SPD)
    ref = OR.rsvd(A, Om, p=rank, q=q, fp16_basis=True)
    A64 = A.astype(np.float64)
    for v in ("tf32", "auto"):
        U, S, V = shg.shg_rsvd(Ad, Od, rank, s, power_iters=q, variant=v)
        S = S.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(S - ref["S"]) / ref["S"]) <= 1e-5, v
        U, V = U.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)
        r_p = np.linalg.norm(A64 - (U * S) @ V.T) / np.linalg.norm(A64)
        assert abs(r_p - ref["r_p"]) <= 0.01 * ref["r_p"], (v, r_p, ref["r_p"])


def test_mode_projections_tf32_and_rp_hosvd_auto(shg):
    """The three mode projections of Algorithm 2 with the TF32 split, and
    RP-HOSVD of a tensor beyond the FP16 range with the automatic variant."""
    dims, J = (64, 48, 40), (12, 9, 16)
    A, _, _ = tucker(dims, (8, 8, 8), seed=3, noise_std=1e-4)
    A = (A.astype(np.float64) * 2.0 ** 20).astype(np.float32)
    oms = hosvd_omegas(dims, J, seed=4)
    X = dev(A)
    for i in range(3):
        om = padded_f16(oms[i])
        W = shg.shg_mode_project(X, om, i, variant="tf32").cpu().numpy()
        ref = OS.project_exact(OH.unfold(A, i), oms[i])
        assert OS.rel_fro_error(W, ref) <= 1e-5, i
    ref = OH.rp_hosvd(A, oms)
    with pytest.raises(shg.ShgError):
        shg.shg_rp_hosvd(X, [padded_f16(o) for o in oms], J, variant="f16")
    core, facs = shg.shg_rp_hosvd(X, [padded_f16(o) for o in oms], J, variant="auto")
    rec = OH.reconstruct(core.cpu().numpy(), [f.cpu().numpy() for f in facs])
    err = np.linalg.norm(A.astype(np.float64) - rec) / np.linalg.norm(A.astype(np.float64))
    assert abs(err - ref["err"]) <= 0.01 * ref["err"], (err, ref["err"])
