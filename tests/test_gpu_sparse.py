"""GPU checks of the sparse sign test matrix (Sec. 3.4): the generator is
bit-exact against the oracle (integer work), and SHGEMM and the randomized SVD
with a sparse Omega match the FP64 oracle at the usual tolerances (the
values -1, 0, 1 are exact in FP16, so the accuracy is that of the split)."""
import numpy as np
import pytest
import torch

from oracle import rsvd as OR
from oracle import shgemm as OS
from oracle import sparse as OSP
from synth import planted_svd, sigma_exp, uniform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shg():
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as m
    return m


def f16_buffer(rows, cols):
    ld = (cols + 7) // 8 * 8
    return torch.empty(rows, ld, dtype=torch.float16, device="cuda")[:, :cols]


@pytest.mark.parametrize("rows,cols,s,seed,offset", [(1000, 64, 3.0, 7, 0), (777, 37, 1.0, 1, 5),
                                                     (2048, 96, 45.25, 9, 1 << 32), (3, 5, 2.0, 0, 0)])
def test_generator_bit_exact(shg, rows, cols, s, seed, offset):
    out = shg.shg_sparse_sign_f16(seed, offset, rows, cols, s, out=f16_buffer(rows, cols))
    got = out.cpu().numpy().astype(np.float64)
    ref = OSP.sparse_sign(seed, offset, rows, cols, s)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("s", [3.0, 32.0])
def test_shgemm_with_sparse_omega(shg, s):
    m, n, k = 513, 1024, 64
    A = uniform(m, n, seed=3)
    Om = OSP.sparse_sign(4, 0, n, k, s)
    Y = shg.shgemm_project(torch.from_numpy(A).cuda(), torch.from_numpy(Om.astype(np.float16)).cuda())
    ref = OS.project_exact(A, Om.astype(np.float16))
    err = OS.rel_fro_error(Y.cpu().numpy(), ref)
    assert err <= 1e-5, err


def test_rsvd_with_sparse_omega(shg):
    m, n, rank, s_over = 1024, 768, 32, 32
    A = planted_svd(m, n, sigma_exp(min(m, n), 8.0), seed=5)
    k = rank + s_over
    Om = OSP.sparse_sign(6, 0, n, k, 3.0).astype(np.float16)
    U, S, V = shg.shg_rsvd(torch.from_numpy(A).cuda(), torch.from_numpy(Om).cuda(), rank=rank, oversampling=s_over)
    ref = OR.rsvd(A, Om, p=rank)
    rel = np.abs(S.cpu().numpy().astype(np.float64) - ref["S"]) / ref["S"]
    assert rel.max() <= 1e-5, rel.max()
