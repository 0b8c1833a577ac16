"""Pins for the FPX codec oracle (Sec. V storage formats): FP32 and the 16-bit format against
library conversions bit for bit, the others against the definition of rounding to nearest with
ties to even, checked by brute force on constructed neighbours."""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

from oracle import fpx


def _wide(rng, n):
    v = rng.standard_normal(n) * 10.0 ** rng.uniform(-46, 39, n)
    edge = [0.0, -0.0, 1e-46, -1e-46, 1.401298464324817e-45, 7e-46, 2.0 ** -149 * 1.5,
            2.0 ** -126, 2.0 ** -126 * (1 - 2.0 ** -30), 3.4028234663852886e38,
            3.4028235677973366e38, 3.4028236e38, 1e39, -1e39, 1.0, -1.5, math.pi]
    return np.concatenate([v, edge])


def test_fp32_matches_ieee_single_bitwise():
    """X = 32 is IEEE FP32: every code equals numpy's round-to-nearest float32 conversion,
    including subnormals, overflow to infinity and signed zeros."""
    rng = np.random.default_rng(0)
    with np.errstate(over="ignore"):
        for v in _wide(rng, 3000):
            ref = struct.unpack("<I", struct.pack("<f", np.float32(v)))[0]
            assert fpx.encode(float(v), 32) == ref, v


def test_fp16_is_bfloat16_bitwise():
    """X = 16 (8 exponent bits, 7 significand bits) is bfloat16: codes equal torch's
    round-to-nearest float32 -> bfloat16 conversion (inputs exact in FP32)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    with np.errstate(over="ignore"):
        x = np.float32(_wide(rng, 3000)).astype(np.float64)
    x = x[np.isfinite(x)]
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).view(torch.int16).numpy().astype(np.uint16)
    got = np.array([fpx.encode(float(v), 16) for v in x], dtype=np.uint16)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("bits", [24, 40, 48, 56])
def test_rounding_to_nearest_ties_to_even_by_brute_force(bits):
    """For random binades, the two FPX neighbours a < b of a point are constructed exactly; a point
    strictly inside rounds to the nearer one, the midpoint to the one with an even code, and both
    neighbours are fixed points of the codec."""
    m = bits - 9
    rng = np.random.default_rng(bits)
    for _ in range(300):
        e = int(rng.integers(-126, 127))
        k = int(rng.integers(0, 1 << m))
        unit = Fraction(2) ** (e - m)
        a = (Fraction(1 << m) + k) * unit
        b = a + unit
        for x, want in ((a + unit / 3, a), (b - unit / 3, b), ((a + b) / 2, None)):
            xf = float(x)
            if Fraction(xf) != x:
                continue  # not an FP64 value
            v = Fraction(fpx.round_value(xf, bits)) if math.isfinite(fpx.round_value(xf, bits)) else None
            if want is None:
                ca, cb = fpx.encode(float(a), bits), fpx.encode(float(b), bits) if b < Fraction(2) ** 128 else None
                even = a if ca % 2 == 0 else b
                if cb is None:
                    continue
                assert v == even
            else:
                assert v == want
        assert fpx.decode(fpx.encode(float(a), bits), bits) == float(a)


@pytest.mark.parametrize("bits", fpx.WIDTHS)
def test_error_bound_monotonicity_and_nesting(bits):
    """|x - round(x)| <= half the spacing; rounding is monotone; every FPX value round-trips
    unchanged through every wider format (the formats nest)."""
    m = bits - 9
    rng = np.random.default_rng(100 + bits)
    x = np.sort(rng.standard_normal(2000) * 10.0 ** rng.uniform(-37, 37, 2000))
    v = np.array([fpx.round_value(float(t), bits) for t in x])
    assert np.all(np.diff(v) >= 0)
    for t, r in zip(x, v):
        e = max(math.frexp(abs(t))[1] - 1, -126)
        assert abs(Fraction(float(t)) - Fraction(float(r))) <= Fraction(2) ** (e - m) / 2
        for wider in fpx.WIDTHS:
            if wider > bits:
                assert fpx.round_value(float(r), wider) == r


@pytest.mark.parametrize("bits", fpx.WIDTHS)
def test_overflow_subnormals_specials(bits):
    m = bits - 9
    largest = float((2 - Fraction(2) ** (-m)) * Fraction(2) ** 127)
    assert fpx.round_value(largest, bits) == largest
    half_ulp = float(Fraction(2) ** (127 - m) / 2)
    assert fpx.round_value(largest + half_ulp, bits) == math.inf   # ties to even: to infinity
    assert fpx.round_value(-(largest + 2 * half_ulp), bits) == -math.inf
    tiny = float(Fraction(2) ** (-126 - m))                           # smallest subnormal
    assert fpx.round_value(tiny, bits) == tiny
    assert fpx.round_value(tiny * 0.49, bits) == 0.0
    assert fpx.round_value(tiny * 0.51, bits) == tiny
    assert fpx.encode(tiny, bits) == 1
    assert fpx.encode(-0.0, bits) == 1 << (bits - 1)
    assert math.isnan(fpx.decode(fpx.encode(math.nan, bits), bits))
    assert fpx.decode(fpx.encode(-math.inf, bits), bits) == -math.inf
    assert fpx.decode(fpx.encode(1.0, bits), bits) == 1.0 and fpx.encode(1.0, bits) == 127 << m


def test_cutoff_and_byte_layout():
    """Magnitudes below the cutoff are stored as +0; codes are X/8 little-endian bytes in order."""
    x = np.array([1e-12, -3e-13, 2.5e-9, -1.0])
    data = fpx.compress(x, 24, cutoff=1e-9)
    assert len(data) == 4 * 3
    out = fpx.decompress(data, 24, 4)
    assert out[0] == 0.0 and out[1] == 0.0 and math.copysign(1.0, out[1]) > 0
    assert out[3] == -1.0 and abs(out[2] - 2.5e-9) <= 2.5e-9 * 2.0 ** -15
    assert data[9:12] == (fpx.encode(-1.0, 24)).to_bytes(3, "little")
    z = np.array([1 + 2j, -3.25 - 0.5j])
    assert np.array_equal(fpx.decompress(fpx.compress(z, 40), 40, 4).view(np.complex128), z)
