"""SHGEMM oracle: Y = A * Omega with FP32 A and FP16 Omega (Sec. 4 of the paper).

Functions
---------
project_exact       the plain definition: A (FP32 values) times Omega (FP16
                    values) in float64.  Each product a*w is exact in float64
                    (24 + 11 significant bits <= 53), so the result is exact up
                    to float64 summation.  Used as C_F64 of the relative error
                    in Sec. 4.4.1.
split_f16           the split of Eqs. shgemm-1 and shgemm-2: hi = toLow(a),
                    lo = toLow((a - toF32(hi)) * 2^11), toLow = FP16 RN-even.
split_tf32          the same split with toLow = TF32 (SHGEMM-TF32, Sec. 4.2:
                    the full FP32 exponent range).
shgemm_emulated     hi*Omega + 2^-11 * lo*Omega (Eq. shgemm-3) in float64,
                    i.e. SHGEMM without any accumulation rounding.
split3_emulated     TCEC-SGEMM (Eq. tcec-5) for two FP32 operands:
                    hiA*hiB + (loA*hiB + hiA*loB) * 2^-11 in float64.
split_bf16          the BF16 analogue with 2 or 3 pieces at scales 2^0, 2^-8,
                    2^-16 (a variant the paper does not print; the same
                    construction as Eq. shgemm-2 with the BF16 unit roundoff).
elementwise_bound   (1/8) n u |A| |Omega| (the SHGEMM bound after Eq.
                    shgemm-ineq, u = 2^-24).
split_bounds        the three inequalities of Eq. split-matrix-ineq.
rel_fro_error       ||C - C_F64||_F / ||C_F64||_F (Sec. 4.4.1).

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from .lowp import FP16, BF16, TF32, round_rn, f16_to_f64

U_FP32 = 2.0 ** -24      # unit roundoff of FP32 (Eq. rounding-error)
U_FP16 = 2.0 ** -11      # unit roundoff of FP16 (after Eq. split-matrix-ineq)


def project_exact(A32: np.ndarray, omega_f16: np.ndarray) -> np.ndarray:
    """Y_ref = A * Omega in float64 (Eq. rp-vec with the Sec. 4.4.1 reference)."""
    A = np.asarray(A32, dtype=np.float32).astype(np.float64)
    W = f16_to_f64(omega_f16)
    return A @ W


def project_exact_t(A32: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A^T * B in float64 (the transposed projection used by the power scheme)."""
    return np.asarray(A32, dtype=np.float32).astype(np.float64).T @ np.asarray(B, dtype=np.float64)


def split_f16(A32: np.ndarray):
    """(hi, lo) of Eqs. shgemm-1, shgemm-2 as float64 arrays of FP16 values.

    hi = RN_f16(a); lo = RN_f16((a - hi) * 2^11).  a - hi is exact (it keeps
    a subset of a's significant bits), and scaling by 2^11 is exact.
    """
    a = np.asarray(A32, dtype=np.float32).astype(np.float64)
    hi = round_rn(a, FP16)
    lo = round_rn((a - hi) * 2.0 ** 11, FP16)
    return hi, lo


def split_tf32(A32: np.ndarray):
    """(hi, lo) of Eqs. shgemm-1 and shgemm-2 with toLow = TF32 (e8m10, RN-even),
    the SHGEMM-TF32 of Sec. 4.2: hi = RN_tf32(a); lo = RN_tf32((a - hi) * 2^11).
    TF32 keeps FP32's exponent range, so no |a| is out of range (only values
    that round past the largest finite TF32 number become infinite)."""
    a = np.asarray(A32, dtype=np.float32).astype(np.float64)
    hi = round_rn(a, TF32)
    lo = round_rn((a - hi) * 2.0 ** 11, TF32)
    return hi, lo


def shgemm_tf32_emulated(A32: np.ndarray, omega_f16: np.ndarray) -> np.ndarray:
    """hi*Omega + 2^-11 * lo*Omega with the TF32 split, float64 (Eq. shgemm-3;
    FP16 Omega values are exact in TF32)."""
    hi, lo = split_tf32(A32)
    W = f16_to_f64(omega_f16)
    return hi @ W + (lo @ W) * 2.0 ** -11


def shgemm_emulated(A32: np.ndarray, omega_f16: np.ndarray) -> np.ndarray:
    """hi*Omega + 2^-11 * lo*Omega in float64 (Eq. shgemm-3, no accumulation error)."""
    hi, lo = split_f16(A32)
    W = f16_to_f64(omega_f16)
    return hi @ W + (lo @ W) * 2.0 ** -11


def split3_emulated(A32: np.ndarray, B32: np.ndarray) -> np.ndarray:
    """TCEC-SGEMM (Eq. tcec-5): hiA*hiB + (loA*hiB + hiA*loB) * 2^-11, float64."""
    ha, la = split_f16(A32)
    hb, lb = split_f16(B32)
    return ha @ hb + (la @ hb + ha @ lb) * 2.0 ** -11


def split_bf16(A32: np.ndarray, pieces: int = 3):
    """BF16 pieces p_0, p_1, ... with a ~= sum_j p_j * 2^(-8 j).

    p_0 = RN_bf16(a); p_j = RN_bf16((a - sum_{i<j} p_i 2^(-8 i)) * 2^(8 j)).
    Each residual is exact in float64.
    """
    a = np.asarray(A32, dtype=np.float32).astype(np.float64)
    out = []
    rem = a.copy()
    for j in range(pieces):
        p = round_rn(rem * 2.0 ** (8 * j), BF16)
        out.append(p)
        rem = rem - p * 2.0 ** (-8 * j)
    return out


def bf16_omega(omega_f16: np.ndarray) -> np.ndarray:
    """RN_bf16 of the FP16 Omega values (float64)."""
    return round_rn(f16_to_f64(omega_f16), BF16)


def shgemm_bf16_emulated(A32: np.ndarray, omega_f16: np.ndarray, pieces: int = 3) -> np.ndarray:
    """sum_j (p_j * Omega_bf16) * 2^(-8 j) in float64."""
    W = bf16_omega(omega_f16)
    ps = split_bf16(A32, pieces)
    return sum((p @ W) * 2.0 ** (-8 * j) for j, p in enumerate(ps))


def elementwise_bound(A32: np.ndarray, omega: np.ndarray, n: int | None = None) -> np.ndarray:
    """(1/8) n u |A| |Omega| with u = 2^-24 (SHGEMM bound, Sec. 4.3)."""
    A = np.abs(np.asarray(A32, dtype=np.float32).astype(np.float64))
    W = np.abs(f16_to_f64(omega) if np.asarray(omega).dtype in (np.uint16, np.float16)
               else np.asarray(omega, dtype=np.float64))
    if n is None:
        n = A.shape[1]
    return (n / 8.0) * U_FP32 * (A @ W)


def split_bounds(A32: np.ndarray):
    """Check the three inequalities of Eq. split-matrix-ineq; returns booleans.

    |A_F16| <= (1+u16)|A|, |dA_F16| <= u16 |A|, |A_delta| <= u16^2 |A|, where
    dA_F16 = lo * 2^-11 and A_delta = A - A_F16 - dA_F16.  The inequalities
    presuppose that A_F16 is an FP16 normal number, |a| >= 2^-14; smaller
    entries (FP16 subnormals) are excluded from the check.
    """
    a32 = np.asarray(A32, dtype=np.float32).astype(np.float64)
    hi, lo = split_f16(A32)
    keep = np.abs(a32) >= 2.0 ** -14
    a = np.abs(a32[keep])
    d = (lo * 2.0 ** -11)[keep]
    rest = a32[keep] - hi[keep] - d
    return (bool(np.all(np.abs(hi[keep]) <= (1 + U_FP16) * a)),
            bool(np.all(np.abs(d) <= U_FP16 * a)),
            bool(np.all(np.abs(rest) <= U_FP16 ** 2 * a)))


def rel_fro_error(C: np.ndarray, C_ref: np.ndarray) -> float:
    """||C - C_ref||_F / ||C_ref||_F (Sec. 4.4.1)."""
    C = np.asarray(C, dtype=np.float64)
    return float(np.linalg.norm(C - C_ref) / np.linalg.norm(C_ref))


def f16_range_ok(A32: np.ndarray) -> bool:
    """True when every |a| rounds to a finite FP16 value (Sec. 4.2: SHGEMM-FP16
    supports only the FP16 exponent range)."""
    hi = round_rn(np.asarray(A32, dtype=np.float32).astype(np.float64), FP16)
    return bool(np.all(np.isfinite(hi)))
