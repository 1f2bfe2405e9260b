"""GPU checks of the projection autotuner: a shape class is timed once and
cached, the cached configuration is used by later projections, and results
under any tuned configuration stay within the SHGEMM tolerance of the FP64
oracle (1e-5 relative Frobenius error; every candidate computes the same
split products, only the staging depths, the drain interval of the hi
product and the CTA grouping differ)."""
import numpy as np
import pytest
import torch

from synth import omega_f16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shg():
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as m
    return m


def rel_err(Y, A, Om):
    ref = A.astype(np.float64) @ Om.astype(np.float64)
    return np.linalg.norm(Y.astype(np.float64) - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("m,n,k", [(2048, 1536, 200), (1000, 776, 64)])
def test_autotune_caches_and_keeps_accuracy(shg, m, n, k):
    shg.shg_autotune_clear()
    rng = np.random.default_rng(m + k)
    A = rng.uniform(-1, 1, size=(m, n)).astype(np.float32)
    Om = omega_f16(n, k, seed=k)
    Ad = torch.from_numpy(A).cuda()
    Od = torch.zeros(n, (k + 7) // 8 * 8, dtype=torch.float16, device="cuda")
    Od[:, :k] = torch.from_numpy(Om).cuda()
    Od = Od[:, :k]
    assert not shg.shg_autotune_lookup(m, n, k)["cached"]
    Y0 = shg.shgemm_project(Ad, Od).cpu().numpy()          # built-in defaults
    cfg = shg.shg_autotune_project(Ad, Od, reps=1)
    assert not cfg["cached"] and cfg["a_stages"] in (2, 4, 6) and cfg["drain_kblocks"] in (2, 4, 8)
    look = shg.shg_autotune_lookup(m, n, k)
    assert look["cached"] and {x: look[x] for x in ("a_stages", "b_stages", "drain_kblocks", "n_groups")} == \
        {x: cfg[x] for x in ("a_stages", "b_stages", "drain_kblocks", "n_groups")}
    # shapes in the same power-of-two buckets of m and n share the entry
    assert shg.shg_autotune_lookup(m + 1, n + 1, k)["cached"]
    assert shg.shg_autotune_project(Ad, Od, reps=1)["cached"]
    Y1 = shg.shgemm_project(Ad, Od).cpu().numpy()          # tuned configuration
    for Y in (Y0, Y1):
        assert rel_err(Y, A, Om) <= 1e-5
    shg.shg_autotune_clear()
    assert not shg.shg_autotune_lookup(m, n, k)["cached"]


def test_batched_autotune_then_batched_rsvd(shg):
    from oracle import rsvd as OR
    from synth import batch_specs, batch_matrix
    shg.shg_autotune_clear()
    specs = batch_specs(5, seed=31, m_range=(300, 700), n_range=(260, 500), ranks=(16, 32))
    As = [batch_matrix(sp) for sp in specs]
    ranks = [sp["rank"] for sp in specs]
    Ad = []
    for A in As:
        r, c = A.shape
        buf = torch.zeros(r, (c + 3) // 4 * 4, dtype=torch.float32, device="cuda")
        buf[:, :c] = torch.from_numpy(A).cuda()
        Ad.append(buf[:, :c])
    tuned = shg.shg_rsvd_batched_autotune(Ad, ranks, 16, seed=7, reps=1)
    assert 1 <= tuned <= len(As)
    assert shg.shg_rsvd_batched_autotune(Ad, ranks, 16, seed=7, reps=1) == 0
    Us, Ss, Vs = shg.shg_rsvd_batched(Ad, ranks, 16, 0, omegas=None, seed=7, use_graph=False)
    # problem 0 against the oracle on the same Philox Omega
    n0, k0 = As[0].shape[1], ranks[0] + 16
    om = shg.shg_gaussian_f16(7, 0, n0, k0, out=torch.empty(n0, (k0 + 7) // 8 * 8, dtype=torch.float16,
                                                           device="cuda")[:, :k0])
    ref = OR.rsvd(As[0], om.cpu().numpy(), p=ranks[0], fp16_basis=True)
    S = Ss[0].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(S - ref["S"]) / ref["S"]) <= 1e-5
    shg.shg_autotune_clear()
