"""GPU checks of the batched randomized SVD (many uneven problems per call):
every problem against the FP64 oracle of Algorithm 1 on the same FP32 A and
FP16 Omega (leading singular values within 1e-5 relative, rank-p residual
within 1 % of the oracle's), generated Omegas against explicitly passed
ones, and CUDA-graph replay against direct launches."""
import numpy as np
import pytest
import torch

from oracle import rsvd as OR
from synth import batch_specs, batch_matrix, omega_f16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shg():
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as m
    return m


def padded_f32(A):
    r, c = A.shape
    buf = torch.zeros(r, (c + 3) // 4 * 4, dtype=torch.float32, device="cuda")
    buf[:, :c] = torch.from_numpy(A).cuda()
    return buf[:, :c]


def padded_f16(Om):
    n, k = Om.shape
    buf = torch.zeros(n, (k + 7) // 8 * 8, dtype=torch.float16, device="cuda")
    buf[:, :k] = torch.from_numpy(Om).cuda()
    return buf[:, :k]


def residual(A, U, S, V):
    A = A.astype(np.float64)
    return np.linalg.norm(A - (U.astype(np.float64) * S.astype(np.float64)) @ V.astype(np.float64).T) / np.linalg.norm(A)


@pytest.fixture(scope="module")
def batch():
    specs = batch_specs(9, seed=21, m_range=(256, 900), n_range=(256, 700), ranks=(16, 32, 48))
    As = [batch_matrix(sp) for sp in specs]
    return specs, As


@pytest.mark.parametrize("q", [0, 1])
@pytest.mark.parametrize("grouped", ["1", "0"])
def test_batched_matches_oracle(shg, batch, q, grouped, monkeypatch):
    """Both execution paths: one grouped launch per step for the whole batch
    (the default), and the per-problem launches on the library's streams
    (SHG_BATCHED_GROUPED=0)."""
    monkeypatch.setenv("SHG_BATCHED_GROUPED", grouped)
    specs, As = batch
    s = 16
    ranks = [sp["rank"] for sp in specs]
    Oms = [omega_f16(A.shape[1], r + s, seed=100 + i) for i, (A, r) in enumerate(zip(As, ranks))]
    Us, Ss, Vs = shg.shg_rsvd_batched([padded_f32(A) for A in As], ranks, s, q,
                                      omegas=[padded_f16(O) for O in Oms], use_graph=False)
    for i, (A, O, r) in enumerate(zip(As, Oms, ranks)):
        ref = OR.rsvd(A, O, p=r, q=q, fp16_basis=True)
        S = Ss[i].cpu().numpy().astype(np.float64)
        rel = np.abs(S - ref["S"]) / ref["S"]
        assert rel.max() <= 1e-5, (i, rel.max())
        r_p = residual(A, Us[i].cpu().numpy(), Ss[i].cpu().numpy(), Vs[i].cpu().numpy())
        assert abs(r_p - ref["r_p"]) <= 0.01 * ref["r_p"], (i, r_p, ref["r_p"])


@pytest.mark.parametrize("grouped", ["1", "0"])
def test_generated_omegas_and_graph_replay(shg, batch, grouped, monkeypatch):
    monkeypatch.setenv("SHG_BATCHED_GROUPED", grouped)
    specs, As = batch
    s = 16
    ranks = [sp["rank"] for sp in specs]
    Ad = [padded_f32(A) for A in As]
    seed = 1234
    # Omega_i is the Philox stream (seed, offset i * 2^32) rounded to FP16
    Oms = [shg.shg_gaussian_f16(seed, i << 32, A.shape[1], r + s,
                                out=torch.empty(A.shape[1], (r + s + 7) // 8 * 8, dtype=torch.float16,
                                                device="cuda")[:, :r + s])
           for i, (A, r) in enumerate(zip(As, ranks))]
    U0, S0, V0 = shg.shg_rsvd_batched(Ad, ranks, s, 0, omegas=Oms, use_graph=False)
    U1, S1, V1 = shg.shg_rsvd_batched(Ad, ranks, s, 0, omegas=None, seed=seed, use_graph=False)
    for a, b in zip(S0, S1):
        assert torch.allclose(a, b, rtol=1e-6, atol=0)
    # graph: captured on the first call, replayed on the second (same buffers)
    out = ([torch.empty_like(u) for u in U0], [torch.empty_like(x) for x in S0], [torch.empty_like(v) for v in V0])
    ws = torch.empty(shg.rsvd_batched_workspace_size([A.shape[0] for A in As], [A.shape[1] for A in As], ranks, s),
                     dtype=torch.uint8, device="cuda")
    flags = shg.new_flags()
    for rep in range(3):
        for t in out[1]:
            t.zero_()
        shg.shg_rsvd_batched(Ad, ranks, s, 0, omegas=None, seed=seed, use_graph=True, out=out, workspace=ws,
                             flags=flags)
        for a, b in zip(S1, out[1]):
            assert torch.allclose(a, b, rtol=1e-6, atol=0), rep


def test_batched_odd_k_and_large_k_grouped(shg):
    """The grouped path with odd k (padded k x k kernels) and k = 144 (the
    panel Cholesky beyond shared memory) in one batch; all singular values
    against the oracle."""
    specs = [dict(m=700, n=600, rate=10.0, rank=17, seed=31), dict(m=900, n=800, rate=20.0, rank=128, seed=32),
             dict(m=513, n=767, rate=8.0, rank=31, seed=33), dict(m=300, n=1000, rate=12.0, rank=64, seed=34)]
    As = [batch_matrix(sp) for sp in specs]
    ranks = [sp["rank"] for sp in specs]
    s = 16
    Oms = [omega_f16(A.shape[1], r + s, seed=200 + i) for i, (A, r) in enumerate(zip(As, ranks))]
    Us, Ss, Vs = shg.shg_rsvd_batched([padded_f32(A) for A in As], ranks, s, 1,
                                      omegas=[padded_f16(O) for O in Oms], use_graph=False)
    for i, (A, O, r) in enumerate(zip(As, Oms, ranks)):
        ref = OR.rsvd(A, O, p=r, q=1, fp16_basis=True)
        S = Ss[i].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(S - ref["S"]) / ref["S"]) <= 1e-5, i
        r_p = residual(A, Us[i].cpu().numpy(), Ss[i].cpu().numpy(), Vs[i].cpu().numpy())
        assert abs(r_p - ref["r_p"]) <= 0.01 * ref["r_p"], (i, r_p, ref["r_p"])
