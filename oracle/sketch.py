"""Learned-sketch oracle: loss, closed-form gradient and the a-posteriori
residual estimator, float64.

The loss of a sketch Omega (n x k) on a matrix A (m x n) is the relative
range-finder residual of Eq. qqta:
    l(Omega) = ||A - Q Q^T A||_F^2 / ||A||_F^2 = 1 - ||Q^T A||_F^2 / ||A||_F^2,
    Q = orth(Y), Y = A Omega.
With P = Q Q^T and M = A A^T, d tr(P M) = 2 tr((I - P) M Y (Y^T Y)^-1 dY^T),
and Y (Y^T Y)^-1 = Q R^-T for Y = Q R, hence
    dl/dY     = -(2 / ||A||_F^2) (I - Q Q^T) A A^T Q R^-T
    dl/dOmega = A^T dl/dY.
The forward pass uses fp16(Omega_master); the gradient with respect to the
FP32 master weights is the gradient with respect to the FP16 values
(straight-through rounding).

A-posteriori estimator (Theorems 1 and 3 of the paper): for a test matrix
G (n x t) with i.i.d. entries of variance alpha,
    E ||(I - Q Q^T) A G||_F^2 = alpha * t * ||(I - Q Q^T) A||_F^2,
so est^2 = ||(I - Q Q^T) A G||_F^2 / (alpha t) is unbiased for the squared
residual; alpha = alpha_Y of the FP16 format for FP16-rounded probes.

Parity unpinned: the gain of a trained sketch over a Gaussian one has no
value printed in the paper; it is measured only.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from .rsvd import qr_pos


def loss(A: np.ndarray, Omega: np.ndarray) -> float:
    A = np.asarray(A, dtype=np.float64)
    Q, _ = qr_pos(A @ np.asarray(Omega, dtype=np.float64))
    nA2 = np.sum(A * A)
    return float(1.0 - np.sum((Q.T @ A) ** 2) / nA2)


def grad_Y(A: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """dl/dY = -(2/||A||^2) (I - Q Q^T) A A^T Q R^-T."""
    A = np.asarray(A, dtype=np.float64)
    Q, R = qr_pos(Y)
    AtQ = A.T @ Q
    M = A @ AtQ                              # A A^T Q
    M = M - Q @ (Q.T @ M)                    # (I - Q Q^T) A A^T Q
    G = np.linalg.solve(R, M.T).T            # M R^-T
    return -2.0 / np.sum(A * A) * G


def grad_omega(A: np.ndarray, Omega: np.ndarray) -> np.ndarray:
    """dl/dOmega = A^T dl/dY."""
    A = np.asarray(A, dtype=np.float64)
    Y = A @ np.asarray(Omega, dtype=np.float64)
    return A.T @ grad_Y(A, Y)


def grad_omega_fd(A: np.ndarray, Omega: np.ndarray, idx, h: float = 1e-6) -> np.ndarray:
    """Central finite differences of ``loss`` at the entries ``idx`` of Omega."""
    Om = np.asarray(Omega, dtype=np.float64)
    out = []
    for (i, j) in idx:
        Op = Om.copy(); Op[i, j] += h
        Omn = Om.copy(); Omn[i, j] -= h
        out.append((loss(A, Op) - loss(A, Omn)) / (2 * h))
    return np.array(out)


def residual_estimate(A: np.ndarray, Q: np.ndarray, G: np.ndarray, alpha: float) -> float:
    """sqrt(||(I - Q Q^T) A G||_F^2 / (alpha t)) / ||A||_F (Theorems 1 and 3)."""
    A = np.asarray(A, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    X = A @ np.asarray(G, dtype=np.float64)
    X = X - Q @ (Q.T @ X)
    t = G.shape[1]
    return float(np.sqrt(np.sum(X * X) / (alpha * t)) / np.linalg.norm(A))
