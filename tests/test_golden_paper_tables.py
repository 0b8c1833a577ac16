"""Values the paper prints in its tables (tests/golden/): Table II's bit counts and rounding
epsilons, which FPX32 / FPX16 must reproduce, and the NR-L device size that the NR-L workload's
block shape follows."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import fpx

HERE = os.path.dirname(os.path.abspath(__file__))


def _table2():
    rows = {}
    with open(os.path.join(HERE, "golden", "table2_bit_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, total, ebits, mbits, eps = line.split()
                rows[name] = (int(total), int(ebits), int(mbits), float(eps))
    return rows


T2 = _table2()


def test_table2_epsilons_are_half_ulps():
    """The printed epsilon of each format is 2^-(significand + 1) to the printed digits."""
    for name, (total, ebits, mbits, eps) in T2.items():
        assert total == 1 + ebits + mbits or name == "TF32", name  # TF32 is a 19-bit format in 32
        assert abs(2.0 ** -(mbits + 1) - eps) / eps < 6e-3, name


@pytest.mark.parametrize("X,name", [(32, "FP32"), (16, "BF16")])
def test_fpx_matches_table2(X, name):
    """FPX32 and FPX16 have the bit counts of FP32 and BF16, and their measured worst relative
    rounding error over many random values reaches that format's epsilon (Table II)."""
    total, ebits, mbits, eps = T2[name]
    assert X == total and X - 9 == mbits and ebits == 8
    rng = np.random.default_rng(7)
    x = rng.uniform(1.0, 2.0, 4000) * 2.0 ** rng.integers(-20, 20, 4000)
    rel = max(abs(fpx.round_value(float(v), X) - v) / v for v in x)
    assert rel <= 2.0 ** -(mbits + 1) and rel > 0.9 * eps


def test_nrl_block_shape_follows_the_device_table():
    """Both nanoribbons tile into whole slices (N_B = orbitals / block size: 6 for NR-S, 10 for
    NR-L), and the NR-L workload uses NR-L's block size and slice count."""
    dev = {}
    with open(os.path.join(HERE, "golden", "nrl_device.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, orbitals, block = line.split()
                dev[name] = (int(orbitals), int(block))
    assert all(o % b == 0 for o, b in dev.values())
    assert dev["NR-S"][0] // dev["NR-S"][1] == 6
    orbitals, block = dev["NR-L"]
    assert W.NRL_CFG["b"] == block
    assert W.NRL_CFG["n_blocks"] == orbitals // block == 10
