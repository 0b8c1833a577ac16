"""Pins for the extended-precision restatement (oracle.hiprec) and its strip fixture.

* its Gauss-Jordan inverse leaves a residual near the extended unit roundoff;
* on the clean strip it reproduces the closed-form integer transmission and the Landauer current;
* where the contacts are well conditioned it agrees with the pinned FP64 oracle to FP64 accuracy;
* the committed fixture (tests/golden/strip_extended.txt) is what the generator computes;
* the FP64 oracle lies within 1e-10 of the fixture on every observable and both energy integrals
  -- the bar the GPU's FP64 path is held to against the same fixture.
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import hiprec as X

HERE = os.path.dirname(os.path.abspath(__file__))
EXT = np.finfo(np.longdouble).nmant >= 63
needs_ext = pytest.mark.skipif(not EXT, reason="no extended long double on this host")


def load_fixture():
    rows = np.loadtxt(os.path.join(HERE, "golden", "strip_extended.txt"))
    nb = W.STRIP_CFG["n_blocks"]
    return dict(energies=rows[:, 0], transmission=rows[:, 1], contact=rows[:, 2:4],
                current=rows[:, 4:4 + nb - 1], density=rows[:, 4 + nb - 1:4 + 2 * nb - 1])


@needs_ext
def test_extended_inverse_residual():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    A[:, 3] = A[:, 2] + 1e-6 * A[:, 3]  # kappa ~ 3e7
    Xi = X._inv(A)
    R = A.astype(X.LD) @ Xi - np.eye(16)
    assert float(np.abs(R).max()) < 16 * np.linalg.cond(A) * 2.0 ** -63


@needs_ext
def test_extended_clean_strip_integer_transmission():
    """T(E) = number of open modes of the clean W = 16 strip (eta = 1e-10), and I_i(E) = T (f_L - f_R)."""
    cfg = W.STRIP_CFG
    s = W.strip(n_blocks=6, disorder=0.0, eta=1e-10, mu_L=cfg["mu_L"], mu_R=cfg["mu_R"], kT=cfg["kT"])
    eps_m = 2 * cfg["t"] * np.cos(np.arange(1, 17) * np.pi / 17)
    for E in (-2.9, -0.05, 0.61, 3.1):
        x = X.rgf_energy(E, s)
        n_open = int(np.sum(np.abs(E - eps_m) < 2))
        assert abs(float(x["transmission"]) - n_open) < 1e-6
        df = O.fermi(E, cfg["mu_L"], cfg["kT"]) - O.fermi(E, cfg["mu_R"], cfg["kT"])
        assert np.abs(x["current"].astype(float) - n_open * df).max() < 1e-6 * max(1, n_open)


@needs_ext
def test_extended_matches_fp64_oracle_where_well_conditioned():
    dev = W.strip(**W.STRIP_CFG)
    idx = [5, 10, 13, 35]  # kappa of the decimation's blocks below 1e3 here
    ref = O.solve(dev, energy_indices=idx, track_cond=True)
    assert np.all(ref["decim_cond"] < 1e3)
    for j, k in enumerate(idx):
        x = X.rgf_energy(float(dev["energies"][k]), dev)
        gr = x["GR_diag"].astype(np.complex128)
        assert np.linalg.norm(ref["GR_diag"][j] - gr) / np.linalg.norm(gr) < 1e-12
        gl = x["GL_diag"].astype(np.complex128)
        assert np.linalg.norm(ref["GL_diag"][j] - gl) / np.linalg.norm(gl) < 1e-12


@needs_ext
def test_fixture_is_what_the_generator_writes():
    fx = load_fixture()
    dev = W.strip(**W.STRIP_CFG)
    assert np.array_equal(fx["energies"], dev["energies"])
    for k in (0, 27, 63):
        x = X.rgf_energy(float(dev["energies"][k]), dev)
        assert np.abs(fx["current"][k] - x["current"].astype(float)).max() <= 1e-15 * np.abs(fx["current"]).max()
        assert np.abs(fx["density"][k] - x["density"].astype(float)).max() <= 1e-15 * np.abs(fx["density"]).max()
        assert abs(fx["transmission"][k] - float(x["transmission"])) <= 1e-15 * max(1.0, abs(fx["transmission"][k]))


def test_fp64_oracle_within_1e10_of_the_fixture():
    """The FP64 oracle (LAPACK inverses) against the extended-precision values: every observable
    within 1e-10 of its largest magnitude over the grid, and both energy integrals within 1e-10.
    (Its G blocks are up to 3.5e-10 off at the energies where the decimation's blocks have condition
    numbers ~3e4 -- at most 141 kappa_dec eps_64 -- which is why blocks are judged with kappa.)"""
    fx = load_fixture()
    dev = W.strip(**W.STRIP_CFG)
    ref = O.solve(dev, keep_blocks=False)
    for k in ("current", "density", "contact", "transmission"):
        r = np.asarray(ref[k]).reshape(64, -1)
        x = np.asarray(fx[k]).reshape(64, -1)
        assert np.abs(r - x).max() < 1e-10 * np.abs(x).max(), k
    w = W.trapezoid_weights(fx["energies"])
    ci, di = w @ fx["current"], (w @ fx["density"]) / (2 * np.pi)
    assert np.abs(ref["current_int"] - ci).max() < 1e-10 * np.abs(ci).max()
    assert np.abs(ref["density_int"] - di).max() < 1e-10 * np.abs(di).max()
