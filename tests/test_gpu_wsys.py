"""GPU parity of the screened-Coulomb (W) system (Table I, W row): assembly of M = I - V P^R and
B^<> = V P^<> V^H on the BT pattern, and the selected solve of M X M^H = B through a system_input
plan, against the oracle (oracle/wsys.py)."""
import numpy as np
import pytest

import workloads as W
from oracle import wsys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2606_25595_gb300 import build
    build.build()
    import paper_2606_25595_gb300 as q
    q.load()
    return q


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _oracle(w):
    out = []
    for k in range(w["n_energies"]):
        PR = (w["PR_diag"][k], w["PR_upper"][k], w["PR_lower"][k])
        M = wsys.assemble(w["V_diag"], w["V_upper"], PR, (w["PL_diag"][k], w["PL_upper"][k]),
                          (w["PG_diag"][k], w["PG_upper"][k]))
        M.update(wsys.solve(M, (M["BL_diag"], M["BL_upper"]), (M["BG_diag"], M["BG_upper"])))
        out.append(M)
    return out


ASSEMBLED = ("M_diag", "M_upper", "M_lower", "BL_diag", "BL_upper", "BG_diag", "BG_upper")
SOLVED = ("XR_diag", "XR_upper", "XR_lower", "XL_diag", "XL_upper", "XG_diag", "XG_upper")


def _check(res, ref, keys, tol):
    worst = 0.0
    for k in keys:
        for e, r in enumerate(ref):
            if r[k].size:
                worst = max(worst, _rel(res[k][e], r[k]))
    assert worst < tol, worst
    return worst


@pytest.mark.parametrize("b,nb,ne,chunk", [(48, 5, 3, 2), (37, 2, 2, 2), (20, 1, 2, 1), (64, 7, 2, 2)])
def test_w_fp64(q, b, nb, ne, chunk):
    """FP64: assembled blocks within 1e-13 and the selected X^R, X^<, X^> within 1e-10 of the
    oracle (kappa(M) ~ 1e2), ragged sizes, one- and two-slice systems, chunked energies."""
    w = W.w_system(b, nb, n_energies=ne, seed=b + nb)
    ref = _oracle(w)
    res = q.solve_w(w, "fp64", max_energies_in_flight=chunk)
    assert np.all(res["status"] == 0)
    _check(res, ref, ASSEMBLED, 1e-13)
    _check(res, ref, SOLVED, 1e-10)


def test_w_emu64(q):
    """Emulated FP64 (tcgen05 digit products) for both the assembly and the solve: X blocks within
    1e-8 (2^-41 products times kappa(M) ~ 1e2 - 1e3)."""
    w = W.w_system(128, 6, n_energies=3, seed=5)
    ref = _oracle(w)
    res = q.solve_w(w, "emu64")
    assert np.all(res["status"] == 0)
    _check(res, ref, ASSEMBLED, 1e-10)
    _check(res, ref, SOLVED, 1e-8)


def test_w_fp32(q):
    """The W system's smaller condition number (Sec. IV) lets complex64 reach kappa * 2^-24: X blocks
    within 1e-4."""
    w = W.w_system(64, 6, n_energies=2, seed=6)
    ref = _oracle(w)
    res = q.solve_w(w, "fp32")
    _check(res, ref, SOLVED, 1e-4)


def test_system_input_validation(q):
    import ctypes
    h = ctypes.c_void_p()
    bad = q.make_desc(4, 16, "fp64", 2, system_input=True, outputs=["GR_diag", "current"])
    assert q.load().qtx_rgf_plan_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    bad = q.make_desc(4, 16, "fp64", 2, system_input=True, has_S=True, outputs=["GR_diag"])
    assert q.load().qtx_rgf_plan_create(ctypes.byref(bad), ctypes.byref(h)) == 1
