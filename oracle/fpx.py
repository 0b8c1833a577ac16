"""FPX storage formats -- test infrastructure only (see the package header).

Sec. V stores the simulation data in custom floating-point formats FPX, X in {56, 48, 40, 32, 24,
16} total bits: one sign bit, the 8-bit exponent and bias (127) of FP32, and X - 9 significand bits,
byte-aligned (X / 8 bytes per value), compressed with IEEE-754 rounding, so that FP32 itself is
one of them bit for bit.  Sec. III adds a value cutoff: magnitudes below it are stored as zero.

Readings (the paper gives no more detail):
  * rounding is IEEE round-to-nearest, ties to even, from the FP64 value; results beyond the
    largest finite FPX value become +-inf, values below the smallest normal use FP32-style
    subnormals (exponent field 0, value q * 2^(-126 - m), m = X - 9);
  * the cutoff applies to |x| before rounding and gives +0;
  * NaN stays NaN (code: positive sign, exponent field all ones, top significand bit set),
    infinities stay infinite, and a result that rounds to zero keeps the sign of x;
  * a value is stored as its X-bit code [sign | exponent | significand] in X / 8 little-endian
    bytes, values one after another.

This module computes the rounding with exact rational arithmetic (fractions.Fraction and
Python's round, which rounds halves to even) rather than with bit manipulation.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

WIDTHS = (56, 48, 40, 32, 24, 16)


def _m(bits: int) -> int:
    if bits not in WIDTHS:
        raise ValueError(f"FPX width must be one of {WIDTHS}")
    return bits - 9


def round_value(x: float, bits: int, cutoff: float = 0.0) -> float:
    """The FPX value nearest to x (ties to even), as a Python float (every FPX value is an FP64
    value).  A result that rounds to zero keeps the sign of x, as in IEEE arithmetic."""
    m = _m(bits)
    if math.isnan(x) or math.isinf(x) or x == 0.0:
        return x
    if abs(x) < cutoff:
        return 0.0
    sign = math.copysign(1.0, x)
    a = Fraction(abs(x))
    # binade 2^e <= a < 2^(e+1); below 2^-126 the spacing stays 2^(-126 - m)
    e = max(math.frexp(abs(x))[1] - 1, -126)
    unit = Fraction(2) ** (e - m)           # spacing of FPX values in this binade
    v = round(a / unit) * unit               # nearest multiple, halves to even
    if v > (2 - Fraction(2) ** (-m)) * Fraction(2) ** 127:
        return sign * math.inf
    return sign * float(v)


def encode(x: float, bits: int, cutoff: float = 0.0) -> int:
    """X-bit code of the FPX value nearest to x."""
    m = _m(bits)
    if math.isnan(x):
        return (0xFF << m) | (1 << (m - 1))
    v = round_value(x, bits, cutoff)
    s = int(math.copysign(1.0, v) < 0)
    if math.isinf(v):
        return (s << (bits - 1)) | (0xFF << m)
    if v == 0.0:
        return s << (bits - 1)
    a = Fraction(abs(v))
    e = math.frexp(abs(v))[1] - 1
    if e < -126:                              # subnormal: q * 2^(-126 - m)
        q = a / Fraction(2) ** (-126 - m)
        assert q.denominator == 1
        return (s << (bits - 1)) | int(q)
    q = a / Fraction(2) ** (e - m) - (1 << m)  # fraction bits below the leading one
    assert q.denominator == 1
    return (s << (bits - 1)) | ((e + 127) << m) | int(q)


def decode(code: int, bits: int) -> float:
    """FP64 value of an X-bit code."""
    m = _m(bits)
    s = -1.0 if (code >> (bits - 1)) & 1 else 1.0
    ef = (code >> m) & 0xFF
    q = code & ((1 << m) - 1)
    if ef == 0xFF:
        return math.nan if q else s * math.inf
    if ef == 0:
        return s * float(Fraction(q) * Fraction(2) ** (-126 - m))
    return s * float((Fraction(1 << m) + q) * Fraction(2) ** (ef - 127 - m))


def compress(x: np.ndarray, bits: int, cutoff: float = 0.0) -> bytes:
    """Little-endian X/8-byte codes of the real values of x (complex arrays: re, im interleaved)."""
    flat = np.ascontiguousarray(x).view(np.float64).ravel() if np.iscomplexobj(x) else \
        np.ascontiguousarray(x, dtype=np.float64).ravel()
    nb = bits // 8
    return b"".join(encode(float(v), bits, cutoff).to_bytes(nb, "little") for v in flat)


def decompress(data: bytes, bits: int, n: int) -> np.ndarray:
    """n FP64 values from their codes."""
    nb = bits // 8
    return np.array([decode(int.from_bytes(data[k * nb:(k + 1) * nb], "little"), bits) for k in range(n)],
                    dtype=np.float64)
