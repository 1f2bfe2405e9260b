"""Low-precision floating point formats eXmY (Sec. 3.1 of the paper).

A format eXmY has X exponent bits, Y explicit mantissa bits, exponent bias
bias(X) = 2^(X-1) - 1 (Sec. 3.2.1), gradual underflow (subnormals) and
IEEE-style overflow to infinity.  Rounding is RN with ties to even, the mode
the paper fixes for the Gaussian values (Sec. 3.1, Eq. RN-range).

The rounding routine works on float64 values: every step (frexp, scaling by
a power of two, np.rint which is round-half-even) is exact in float64 for the
formats used here (Y <= 23), so the result is the correctly rounded value.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


class Fmt:
    """eXmY descriptor (Sec. 3.1)."""

    def __init__(self, name: str, X: int, Y: int):
        self.name, self.X, self.Y = name, X, Y
        self.bias = 2 ** (X - 1) - 1                       # bias(X), Sec. 3.2.1
        self.emin = 1 - self.bias                          # exponent of min normal
        self.emax = 2 ** X - 2 - self.bias                 # largest finite exponent
        self.min_normal = 2.0 ** self.emin                 # 0b0'00..01'00..0
        self.min_subnormal = 2.0 ** (self.emin - Y)        # 0b0'00..00'00..01
        self.max_finite = (2.0 - 2.0 ** (-Y)) * 2.0 ** self.emax
        self.u = 2.0 ** (-(Y + 1))                         # unit roundoff u_Y

    def __repr__(self):
        return f"Fmt({self.name}, e{self.X}m{self.Y})"


FP8_E4M3 = Fmt("fp8_e4m3", 4, 3)
FP8_E5M2 = Fmt("fp8_e5m2", 5, 2)
FP16 = Fmt("fp16", 5, 10)
BF16 = Fmt("bf16", 8, 7)
TF32 = Fmt("tf32", 8, 10)
FP32 = Fmt("fp32", 8, 23)


def round_rn(x, fmt: Fmt) -> np.ndarray:
    """RN-even rounding of float64 values to the eXmY format ``fmt``.

    Returns float64 values that are exactly representable in ``fmt``; values
    whose rounded magnitude exceeds the largest finite number become +-inf.
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    fin = np.isfinite(x) & (x != 0)
    xf = x[fin]
    _, e = np.frexp(xf)                 # xf = f * 2^e, 0.5 <= |f| < 1
    e = e - 1                           # xf = g * 2^e, 1 <= |g| < 2
    e = np.maximum(e, fmt.emin)         # subnormal range shares the min exponent
    q = np.ldexp(1.0, e - fmt.Y)        # quantum (ulp) at that exponent
    r = np.rint(xf / q) * q             # xf/q exact; rint = round half to even
    r[np.abs(r) > fmt.max_finite] = np.inf * np.sign(r[np.abs(r) > fmt.max_finite])
    out[fin] = r
    out[~np.isfinite(x)] = x[~np.isfinite(x)]
    return out


def decode_bits(bits, fmt: Fmt) -> np.ndarray:
    """Value of the eXmY bit pattern(s) ``bits`` (sign | exponent | mantissa)."""
    b = np.asarray(bits, dtype=np.int64)
    sign = np.where((b >> (fmt.X + fmt.Y)) & 1, -1.0, 1.0)
    ef = (b >> fmt.Y) & ((1 << fmt.X) - 1)
    mf = (b & ((1 << fmt.Y) - 1)).astype(np.float64)
    normal = sign * np.ldexp(1.0 + mf * 2.0 ** (-fmt.Y), ef - fmt.bias)
    sub = sign * np.ldexp(mf, fmt.emin - fmt.Y)
    val = np.where(ef == 0, sub, normal)
    special = ef == (1 << fmt.X) - 1
    val = np.where(special & (mf == 0), sign * np.inf, val)
    val = np.where(special & (mf != 0), np.nan, val)
    return val


def all_finite_values(fmt: Fmt) -> np.ndarray:
    """Every finite value of ``fmt`` (both zeros included), by enumeration."""
    nbits = 1 + fmt.X + fmt.Y
    v = decode_bits(np.arange(1 << nbits, dtype=np.int64), fmt)
    return v[np.isfinite(v)]


def f16_to_f64(omega_f16) -> np.ndarray:
    """Exact float64 values of FP16 data given as float16 or uint16 bits."""
    a = np.asarray(omega_f16)
    if a.dtype == np.uint16:
        return decode_bits(a.astype(np.int64), FP16)
    return a.astype(np.float64)


def bf16_to_f64(bits) -> np.ndarray:
    """Exact float64 values of BF16 data given as uint16 bits."""
    return decode_bits(np.asarray(bits).astype(np.int64), BF16)


def encode_bf16(x) -> np.ndarray:
    """uint16 bit patterns of values already representable in BF16."""
    x32 = np.asarray(x, dtype=np.float32)
    return (x32.view(np.uint32) >> 16).astype(np.uint16)
