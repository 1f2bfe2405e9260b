"""Sparse sign test matrices (Sec. 3.4; Eq. sp-rand of Sec. 2.2 without the
sqrt(s) factor, which the range finder does not need).

Element (r, c) of a rows x cols matrix, e = r * cols + c, takes 32-bit word
e mod 4 of the Philox4x32-10 block (e div 4) + offset under key (seed lo,
seed hi) -- the same stream as the Gaussian test matrix -- and becomes
    +1 if w < T,   -1 if w >= 2^32 - T,   0 otherwise,
with T = floor(2^32 / (2 s) + 1/2) (at most 2^31), so that
P(+1) = P(-1) = T / 2^32 ~ 1 / (2 s) and P(0) ~ 1 - 1/s.
s = 1 gives Rademacher signs, s = 3 Achlioptas' matrix, s = sqrt(n) Li et
al.'s very sparse matrix.  All three values are exact in FP16.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import math

import numpy as np

from .gaussian import philox4x32_10


def threshold(s: float) -> int:
    """T = floor(2^32 / (2 s) + 1/2), capped at 2^31 (s >= 1)."""
    if not s >= 1.0:
        raise ValueError("s must be >= 1")
    return min(2 ** 31, int(math.floor(2.0 ** 32 / (2.0 * s) + 0.5)))


def philox_words(seed: int, offset: int, count: int) -> np.ndarray:
    """The first `count` 32-bit words of the stream: word e = component e % 4
    of block e // 4 + offset."""
    nblk = (count + 3) // 4
    b = np.arange(nblk, dtype=np.uint64) + np.uint64(offset)
    ctr = np.stack([b & np.uint64(0xFFFFFFFF), b >> np.uint64(32),
                    np.zeros_like(b), np.zeros_like(b)], axis=-1)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    return philox4x32_10(ctr, key).reshape(-1)[:count]


def sparse_sign(seed: int, offset: int, rows: int, cols: int, s: float) -> np.ndarray:
    """rows x cols matrix of {-1, 0, +1} (float64)."""
    t = threshold(s)
    w = philox_words(seed, offset, rows * cols).astype(np.uint64)
    out = np.zeros(rows * cols)
    out[w < np.uint64(t)] = 1.0
    out[w >= np.uint64(2 ** 32 - t)] = -1.0
    return out.reshape(rows, cols)
