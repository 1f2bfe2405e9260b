"""CPU study of the accuracy of the random projection with low-precision
Gaussian test matrices (the numerical experiment closing the analysis of
Sec. 3).  Test infrastructure only.

The Gaussian matrix G (n x k) is drawn in FP32 and rounded RN to a shorter
mantissa (an eXmY format of `oracle.lowp`), then A and G are taken to FP64
and the projection error ||A - Q Q^T A||_F with Q = orth(A G) is computed in
FP64, so that only the rounding of G differs between formats.

Input matrices (both n x n, after the test matrices the paper adopts):
* Type 1: A = diag(I_r, 0) + (xi / n) G_A G_A^T with G_A Gaussian.  The
  paper prints the factor as xi over epsilon; it is read as xi / n (the
  source's noise level relative to the matrix size; with machine epsilon the
  noise term would exceed the signal by eleven orders of magnitude).
* Type 2: A = U D V^T with Haar U, V and
  D = diag(phi I_r, 2^-alpha, 3^-alpha, ..., (n - r + 1)^-alpha).
The paper fixes n = 4096, r = 20, xi = 1e-4, alpha = 3, phi = 1e6 and does
not print k; the study uses k = r + 10.

    python -m oracle.mantissa_study [n]        # the paper's n = 4096 by default
"""
from __future__ import annotations

import sys

import numpy as np

from .lowp import BF16, FP8_E4M3, FP8_E5M2, FP16, Fmt, round_rn

# e8mY: FP32's exponent range with Y mantissa bits; FP8/FP16/BF16 with their own
FORMATS = [Fmt("e8m23", 8, 23), Fmt("e8m10", 8, 10), FP16, BF16, FP8_E4M3, FP8_E5M2, Fmt("e8m2", 8, 2),
           Fmt("e8m1", 8, 1)]


def haar(n: int, rng) -> np.ndarray:
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(R))


def type1(n: int, r: int, xi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    A = (xi / n) * (G @ G.T)
    A[np.arange(r), np.arange(r)] += 1.0
    return A.astype(np.float32)


def type2(n: int, r: int, alpha: float, phi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    d = np.concatenate([np.full(r, phi), np.arange(2, n - r + 2, dtype=np.float64) ** (-alpha)])
    U = haar(n, rng)
    V = haar(n, rng)
    return ((U * d) @ V.T).astype(np.float32)


def projection_error(A32: np.ndarray, G: np.ndarray) -> float:
    """||A - Q Q^T A||_F in FP64, Q an orthonormal basis of range(A G)."""
    A = np.asarray(A32, dtype=np.float64)
    Q, _ = np.linalg.qr(A @ np.asarray(G, dtype=np.float64))
    return float(np.linalg.norm(A - Q @ (Q.T @ A)))


def study(A32: np.ndarray, k: int, seed: int, formats=FORMATS) -> dict:
    """Projection error for G drawn in FP32 (seed) and rounded to each format."""
    n = A32.shape[1]
    G32 = np.random.default_rng(seed).standard_normal((n, k)).astype(np.float32).astype(np.float64)
    return {f.name: projection_error(A32, round_rn(G32, f)) for f in formats}


def main(n: int = 4096) -> None:
    r, k = 20, 30
    for name, A in (("type1", type1(n, r, 1e-4, seed=1)), ("type2", type2(n, r, 3.0, 1e6, seed=2))):
        res = study(A, k, seed=10)
        base = res["e8m23"]
        print(name, " ".join(f"{f}={e / base:.4f}" for f, e in res.items()), f"(e8m23 error {base:.4e})")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 4096)
