"""GPU check of the Gram matrix G = X^T X, the first step of each CholeskyQR
pass (the orthonormal basis of Algorithms 1 and 2).

The library sums the exact FP32 products with compensated FP32 arithmetic in
128-row blocks that meet in FP64.  The bound of the compensated dot product
(Ogita, Rump and Oishi 2005) for a block of n = 128 terms is
gamma_n^2 sum |x_ri x_rj| with gamma_n = n u / (1 - n u), u = 2^-24, i.e.
about 5.8e-11 (|X|^T |X|)_ij; the reference is numpy's FP64 product of the
same FP32 values (error below m 2^-53 (|X|^T |X|)_ij).  Plain FP32 sums would
miss the bound by orders of magnitude, so the test also shows that the
compensation works.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


@pytest.fixture(scope="module")
def shg():
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as m
    return m


def graded(m, k, seed):
    """Columns of mixed sign and magnitudes spread over 2^-12 .. 2^0."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, k)) * 2.0 ** (-12.0 * rng.random(k))
    return X.astype(np.float32)


@pytest.mark.parametrize("m,k", [(1, 1), (31, 5), (1000, 33), (4099, 64), (4096, 266), (20000, 130)])
def test_gram_within_compensated_bound(shg, m, k):
    X = graded(m, k, seed=m + k)
    ldx = (k + 3) // 4 * 4
    buf = torch.zeros(m, ldx, dtype=torch.float32, device="cuda")
    buf[:, :k] = torch.from_numpy(X).cuda()
    G = shg.shg_gram(buf[:, :k]).cpu().numpy()
    X64 = X.astype(np.float64)
    ref = X64.T @ X64
    absref = np.abs(X64).T @ np.abs(X64)
    iu = np.triu_indices(k)
    gam = 128 * U / (1 - 128 * U)
    bound = gam * gam * absref + m * 2.0 ** -53 * absref
    err = np.abs(G - ref)
    assert np.all(err[iu] <= bound[iu]), float(np.max(err[iu] / absref[iu]))
    assert np.all(G[np.tril_indices(k, -1)] == 0.0)


def test_gram_rejects_bad_arguments(shg):
    X = torch.zeros(8, 4, device="cuda")
    with pytest.raises(ValueError):
        shg.shg_gram(X, out=torch.empty(3, 3, dtype=torch.float64, device="cuda"))
