"""Low-precision Gaussian values (Sec. 3 of the paper) and the counter-based
generator the GPU path also implements.

Table 1 quantities
------------------
p_overflow, p_underflow, p_not_normalized    Sec. 3.2.1, Table 1 (top)
count_within(fmt, s)                          Sec. 3.2.2, Table 1 (bottom), by enumeration
count_within_formula(fmt, s)                  the closed form the printed table satisfies
alpha_Y(fmt)                                  Sec. 3.2.3, variance of RN-rounded N(0,1)

Readings (the printed text is garbled here):
* Phi is the N(0,1) cumulative distribution (the text calls it a density).
* The printed probabilities p_uf and p_not-normalized match
  2 * (Phi(t/2) - 1/2) with t = min_denormalized resp. min_normalized, not
  2 * (Phi(t) - 1/2) as printed; for p_uf t/2 is exactly the RN boundary
  below which a value rounds to zero.  We reproduce the table with t/2.
* The printed closed form of N^{2^s sigma} (2(s+bias+1)2^Y + 1) does not
  match the printed table; the table equals the number of finite values in
  the open interval (-2^s, 2^s), which is 2 (s + bias) 2^Y - 1.
* The alpha_Y sum has a misplaced parenthesis; alpha_Y is the sum over all
  values v of v^2 times the probability that RN rounds N(0,1) to v.

Counter-based generator
-----------------------
philox4x32_10   Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
                as 1, 2, 3", SC'11: 10 rounds of the Philox-4x32 bijection.
box_muller      the standard Box-Muller transform of two uniforms.
gaussian_f16    Omega[r, c] as the GPU path defines it: element e = r*cols + c
                of the stream takes normal (e mod 4) of Philox block e div 4
                (+ offset), then RN to FP16.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import ndtr

from .lowp import Fmt, FP16, round_rn, all_finite_values


# ----------------------------------------------------------------- Table 1

def p_overflow(fmt: Fmt) -> float:
    """P(|g| > max) = 2 (1 - Phi(max_eXmY)) (Sec. 3.2.1)."""
    return float(2.0 * (1.0 - ndtr(fmt.max_finite)))


def p_underflow(fmt: Fmt) -> float:
    """Probability that RN rounds N(0,1) to zero: 2 (Phi(min_sub / 2) - 1/2)."""
    return float(2.0 * (ndtr(fmt.min_subnormal / 2.0) - 0.5))


def p_not_normalized(fmt: Fmt) -> float:
    """Table 1's 'denormalized or underflowed' column: 2 (Phi(min_normal / 2) - 1/2)."""
    return float(2.0 * (ndtr(fmt.min_normal / 2.0) - 0.5))


def count_within(fmt: Fmt, s: int) -> int:
    """Number of finite eXmY values v with |v| < 2^s, by enumeration (Sec. 3.2.2)."""
    v = all_finite_values(fmt)
    v = np.unique(v)                    # +0 and -0 are one value
    return int(np.count_nonzero(np.abs(v) < 2.0 ** s))


def count_within_formula(fmt: Fmt, s: int) -> int:
    """2 (s + bias(X)) 2^Y - 1 (the value Table 1 prints)."""
    return 2 * (s + fmt.bias) * 2 ** fmt.Y - 1


def alpha_Y(fmt: Fmt) -> float:
    """E[g_eXmY^2] for g ~ N(0,1) rounded RN to eXmY (Sec. 3.2.3).

    Each finite value v receives the probability mass of its RN bucket,
    whose edges are the midpoints to the neighbouring values.
    """
    v = np.unique(all_finite_values(fmt))
    v = v[v >= 0]                        # symmetric: sum over v >= 0, doubled
    lo = np.empty_like(v)
    hi = np.empty_like(v)
    lo[1:] = 0.5 * (v[1:] + v[:-1])
    lo[0] = 0.0
    hi[:-1] = lo[1:]
    # the largest finite value keeps everything up to its overflow threshold
    hi[-1] = v[-1] + 0.5 * (v[-1] - v[-2])
    mass = ndtr(hi) - ndtr(lo)
    return float(2.0 * np.sum(v * v * mass))


# ------------------------------------------------------------ Philox4x32-10

_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox-4x32 with 10 rounds (SC'11).  ctr: (..., 4) uint32, key: (..., 2).

    One round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (64-bit products),
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); then the key is bumped by
    the Weyl constants (W0, W1).  Vectorised over leading dimensions.
    """
    c = np.array(ctr, dtype=np.uint64) & _MASK
    k = np.array(key, dtype=np.uint64) & _MASK
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for _ in range(10):
        p0 = c0 * np.uint64(_M0)
        p1 = c2 * np.uint64(_M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(_MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(_MASK)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(_W0)) & np.uint64(_MASK)
        k1 = (k1 + np.uint64(_W1)) & np.uint64(_MASK)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def uniform_open01(x_u32) -> np.ndarray:
    """Map a 32-bit integer to (0, 1): (x + 1/2) * 2^-32, in float64."""
    return (np.asarray(x_u32, dtype=np.float64) + 0.5) * 2.0 ** -32


def box_muller(u1, u2):
    """(sqrt(-2 ln u1) cos(2 pi u2), sqrt(-2 ln u1) sin(2 pi u2)), float64."""
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)


def gaussian_f64(seed: int, offset: int, rows: int, cols: int) -> np.ndarray:
    """N(0,1) matrix (float64, before rounding) of the counter-based stream."""
    n = rows * cols
    nblk = (n + 3) // 4
    blk = np.arange(nblk, dtype=np.uint64) + np.uint64(offset)
    ctr = np.stack([blk & np.uint64(_MASK), blk >> np.uint64(32),
                    np.zeros_like(blk), np.zeros_like(blk)], axis=-1)
    key = np.array([seed & _MASK, (seed >> 32) & _MASK], dtype=np.uint64)
    x = philox4x32_10(ctr, key)
    z0, z1 = box_muller(uniform_open01(x[:, 0]), uniform_open01(x[:, 1]))
    z2, z3 = box_muller(uniform_open01(x[:, 2]), uniform_open01(x[:, 3]))
    z = np.stack([z0, z1, z2, z3], axis=-1).reshape(-1)[:n]
    return z.reshape(rows, cols)


def gaussian_f16(seed: int, offset: int, rows: int, cols: int) -> np.ndarray:
    """The same stream rounded RN-even to FP16 values (float64 array)."""
    return round_rn(gaussian_f64(seed, offset, rows, cols), FP16)
