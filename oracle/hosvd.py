"""Random-projection HOSVD oracle (Algorithm 2 of the paper, Sec. 5.2), float64.

For each mode i:  W <- A_(i) Omega_(i);  Q_i <- QR(W)   (diag(R) > 0)
then the core     g <- A x_1 Q_1^T x_2 Q_2^T ... x_N Q_N^T
and the approximation A ~ g x_1 Q_1 ... x_N Q_N.

Readings (the printed text is inconsistent about Q_i vs Q_i^T in the mode
products; these are pinned with explicit indices):
* A is stored row-major, last index fastest.  The unfolding A_(i) has the
  mode-i index as its row and, as its column, the row-major linear index of
  the remaining indices with index i deleted.  For a 3-way tensor and mode 2
  the column of A[i1, i2, i3] is i1 * I3 + i3.
* Omega_(i) has prod_{j != i} I_j rows in that column order and J_i columns,
  where J_i = r_i + s includes the oversampling (Algorithm 3 shows the ranks
  J_i include padding).  Q_i keeps all J_i columns.
* core g[j1, .., jN] = sum_{i1..iN} A[i1, .., iN] Q_1[i1, j1] ... Q_N[iN, jN];
  reconstruction A_hat[i1, .., iN] = sum_j g[j] Q_1[i1, j1] ... Q_N[iN, jN].

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from .lowp import f16_to_f64
from .rsvd import qr_pos


def unfold(A: np.ndarray, i: int) -> np.ndarray:
    """A_(i): rows = mode-i index, columns = row-major index of the other modes."""
    return np.moveaxis(A, i, 0).reshape(A.shape[i], -1)


def mode_product_T(T: np.ndarray, Q: np.ndarray, i: int) -> np.ndarray:
    """(T x_i Q^T)[.., j, ..] = sum_a T[.., a, ..] Q[a, j]."""
    return np.moveaxis(np.tensordot(T, Q, axes=([i], [0])), -1, i)


def mode_product(T: np.ndarray, Q: np.ndarray, i: int) -> np.ndarray:
    """(T x_i Q)[.., a, ..] = sum_j T[.., j, ..] Q[a, j]."""
    return np.moveaxis(np.tensordot(T, Q, axes=([i], [1])), -1, i)


def rp_hosvd(A32: np.ndarray, omegas) -> dict:
    """Algorithm 2.  omegas[i]: (prod_{j!=i} I_j) x J_i FP16 (or float64)."""
    A = np.asarray(A32, dtype=np.float32).astype(np.float64)
    Qs, Ws = [], []
    for i in range(A.ndim):
        om = np.asarray(omegas[i])
        Om = f16_to_f64(om) if om.dtype in (np.float16, np.uint16) else om.astype(np.float64)
        W = unfold(A, i) @ Om
        Q, _ = qr_pos(W)
        Ws.append(W)
        Qs.append(Q)
    g = A
    for i in range(A.ndim):
        g = mode_product_T(g, Qs[i], i)
    Ahat = g
    for i in range(A.ndim):
        Ahat = mode_product(Ahat, Qs[i], i)
    err = float(np.linalg.norm(A - Ahat) / np.linalg.norm(A))
    return dict(W=Ws, Q=Qs, core=g, err=err)


def reconstruct(core: np.ndarray, Qs) -> np.ndarray:
    """g x_1 Q_1 x_2 Q_2 ... (float64)."""
    T = np.asarray(core, dtype=np.float64)
    for i, Q in enumerate(Qs):
        T = mode_product(T, np.asarray(Q, dtype=np.float64), i)
    return T
