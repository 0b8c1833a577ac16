"""The FPX format parameters the paper states (tests/golden/fpx_formats.txt, Sec. V) against the
FPX oracle's codes and the library's byte count (qtx_fpx_bytes, no GPU needed)."""
import math
import os

import numpy as np
import pytest

from oracle import fpx

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    rows = []
    with open(os.path.join(HERE, "golden", "fpx_formats.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


ROWS = _rows()


def test_fixture_covers_the_papers_widths():
    assert tuple(r[0] for r in ROWS) == fpx.WIDTHS


@pytest.mark.parametrize("X,ebits,bias,mbits,nbytes", ROWS)
def test_oracle_code_layout(X, ebits, bias, mbits, nbytes):
    """1.0 has the biased exponent in the field above mbits significand bits and a zero
    significand; -0 sets only the top (sign) bit; the largest finite value is (2 - 2^-m) 2^(2^e -
    2 - bias) with every exponent bit but the last and every significand bit set."""
    assert X == 1 + ebits + mbits
    assert fpx.encode(1.0, X) == bias << mbits
    assert fpx.encode(-0.0, X) == 1 << (X - 1)
    top = (2 - 2.0 ** -mbits) * 2.0 ** ((1 << ebits) - 2 - bias)
    assert fpx.encode(top, X) == (((1 << ebits) - 2) << mbits) | ((1 << mbits) - 1)
    assert fpx.decode(fpx.encode(top, X), X) == top
    assert math.isinf(fpx.round_value(top * (1 + 2.0 ** -mbits), X))
    # one value per X / 8 bytes
    assert len(fpx.compress(np.array([1.0, -2.5, 3e-5]), X)) == 3 * nbytes


@pytest.mark.parametrize("X,ebits,bias,mbits,nbytes", ROWS)
def test_library_byte_count(X, ebits, bias, mbits, nbytes):
    q = pytest.importorskip("paper_2606_25595_gb300")
    try:
        lib = q.load()
    except Exception as exc:  # the library must be built first (build() compiles it here too)
        pytest.skip(f"library not built: {exc}")
    assert lib.qtx_fpx_bytes(X, 1000) == 1000 * nbytes
