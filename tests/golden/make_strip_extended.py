"""Writes strip_extended.txt: the config-1 strip's observables (W = 16, b = 16, N_B = 32, 64 energies on
[-3.5, 3.5], eta = 1e-6, contacts by decimation) from the extended-precision restatement of the
selected solve, ``oracle.hiprec`` (numpy clongdouble: 64-bit significands on x86), so that FP64 results
can be judged by their distance from the exact values rather than from another FP64 evaluation.

Run from the repository root:  python tests/golden/make_strip_extended.py
Calls only ``oracle`` (and ``workloads`` for the seeded inputs)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import hiprec  # noqa: E402


def main():
    assert np.finfo(np.longdouble).nmant >= 63, "needs an extended long double (x86 80-bit or quad)"
    dev = W.strip(**W.STRIP_CFG)
    lines = ["# Config-1 strip (workloads.STRIP_CFG, seed 0) from oracle.hiprec in extended precision",
             "# (np.clongdouble, %d-bit significand), written by tests/golden/make_strip_extended.py." %
             (np.finfo(np.longdouble).nmant + 1),
             "# One line per energy: E, transmission, contact_L, contact_R, current[0..30], density[0..31]"]
    for E in dev["energies"]:
        x = hiprec.rgf_energy(float(E), dev)
        vals = [float(E), float(x["transmission"]), *[float(v) for v in x["contact"]],
                *[float(v) for v in x["current"]], *[float(v) for v in x["density"]]]
        lines.append(" ".join(repr(v) for v in vals))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "strip_extended.txt")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(out)


if __name__ == "__main__":
    main()
