"""Randomized SVD oracle (Algorithm 1 of the paper, Sec. 2.1-2.2), float64.

Algorithm 1 with the power scheme of Sec. 2.1:
    Y <- A Omega                                     (Eq. rp-vec)
    Q, R <- QR(Y)                                    (Householder, diag(R) > 0)
    repeat q times:  Z <- orth(A^T Q);  Q <- orth(A Z)   (A_hat = (A A^T)^q A)
    B <- Q^T A
    U', Sigma_1, V <- tSVD(B, rank p)
    U <- Q U'

Readings (the paper is silent on these points):
* QR is made unique by requiring diag(R) > 0; CholeskyQR produces exactly
  that factor, Householder QR matches it after a sign flip per column.
* The power scheme is orthonormalised after every product (the numerically
  stable form of (A A^T)^q A Omega).  With ``fp16_basis=True`` the basis is
  rounded to FP16 before each projection, so that each projection is itself
  an SHGEMM whose FP16 operand is the current basis; the FP16 basis acts as a
  new test matrix.
* Singular vectors are unique up to sign; ``canonical_signs`` makes the
  largest-magnitude entry of each left vector positive.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from .lowp import FP16, round_rn, f16_to_f64


def qr_pos(Y: np.ndarray):
    """Thin Householder QR with diag(R) > 0 (unique factor)."""
    Q, R = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s, R * s[:, None]


def canonical_signs(U: np.ndarray, V: np.ndarray | None = None):
    """Flip column signs so that each column of U has its largest-|.| entry > 0."""
    idx = np.argmax(np.abs(U), axis=0)
    s = np.sign(U[idx, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return (U * s, None if V is None else V * s)


def rsvd(A32: np.ndarray, omega: np.ndarray, p: int, q: int = 0, fp16_basis: bool = False):
    """Algorithm 1.  A32: m x n FP32 values; omega: n x k FP16 (float16/uint16)
    or float64 values.  Returns a dict with Y, Q, B, U (m x p), S (p), V (n x p)
    and the residuals r_p = ||A - U S V^T||_F/||A||_F and
    r_k = ||A - Q Q^T A||_F/||A||_F."""
    A = np.asarray(A32, dtype=np.float32).astype(np.float64)
    om = np.asarray(omega)
    W = f16_to_f64(om) if om.dtype in (np.float16, np.uint16) else om.astype(np.float64)
    Y = A @ W                                    # projection
    Q, _ = qr_pos(Y)                             # orthonormal basis
    for _ in range(q):                           # power scheme, Sec. 2.1
        Qb = round_rn(Q, FP16) if fp16_basis else Q
        Z, _ = qr_pos(A.T @ Qb)
        Zb = round_rn(Z, FP16) if fp16_basis else Z
        Q, _ = qr_pos(A @ Zb)
    B = Q.T @ A                                  # B = Q^T A
    Ub, S, Vt = np.linalg.svd(B, full_matrices=False)   # small SVD of B
    U = Q @ Ub[:, :p]                            # lift the left vectors
    V = Vt[:p].T
    U, V = canonical_signs(U, V)
    S = S[:p]
    nA = np.linalg.norm(A)
    r_p = np.linalg.norm(A - (U * S) @ V.T) / nA
    r_k = np.linalg.norm(A - Q @ (Q.T @ A)) / nA
    return dict(Y=Y, Q=Q, B=B, U=U, S=S, V=V, r_p=float(r_p), r_k=float(r_k),
                S_all=np.linalg.svd(B, compute_uv=False))


def eckart_young(sigma_all: np.ndarray, p: int, normA: float | None = None) -> float:
    """||Sigma_2||_F (/||A||_F if given): the best rank-p residual (Theorem Eckart-Young)."""
    s = np.asarray(sigma_all, dtype=np.float64)
    r = float(np.sqrt(np.sum(s[p:] ** 2)))
    return r / normA if normA else r


def halko_bound(sigma_all: np.ndarray, p: int, s: int) -> float:
    """sqrt(1 + p/(s-1)) ||Sigma_2||_F (Eq. qqta-acc, rank p, oversampling s)."""
    return float(np.sqrt(1.0 + p / (s - 1.0)) * eckart_young(sigma_all, p))
