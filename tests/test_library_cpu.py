"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every function that
include/*.h declares.  No compute call is made (there is no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(qtx_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_25595_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for fn in ("qtx_rgf_plan_create", "qtx_rgf_solve", "qtx_rgf_destroy"):
        assert fn in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_lists_the_exports(libpath):
    import paper_2606_25595_gb300 as q
    assert set(q.EXPORTED) <= set(_declared_functions())
    assert q.load().qtx_rgf_version().decode().startswith("qtx-rgf")


def test_footprint_and_validation(libpath):
    import paper_2606_25595_gb300 as q
    d = q.make_desc(64, 256, "fp64", max_energies_in_flight=8)
    fp = q.footprint(d)
    # g and g^< alone: 2 * N_B * Ec * b^2 * 16 bytes
    assert fp >= 2 * 64 * 8 * 256 * 256 * 16
    d32 = q.make_desc(64, 256, "fp32", max_energies_in_flight=8)
    assert q.footprint(d32) < fp
    bad = q.make_desc(0, 16)
    assert q.footprint(bad) == 0
    h = ctypes.c_void_p()
    s = q.load().qtx_rgf_plan_create(ctypes.byref(bad), ctypes.byref(h))
    assert s == 1 and not h.value
    assert b"n_blocks" in q.load().qtx_rgf_last_error(None)


def test_block_tridiagonal_sigma_descriptor(libpath):
    """offdiag_sigma needs has_scattering; it adds two b x b work blocks per energy, and per-energy
    U, V blocks when the off-diagonal self-energies depend on the energy."""
    import paper_2606_25595_gb300 as q
    h = ctypes.c_void_p()
    bad = q.make_desc(8, 32, "fp64", 4, has_scattering=False, offdiag_sigma=True)
    assert q.load().qtx_rgf_plan_create(ctypes.byref(bad), ctypes.byref(h)) == 1 and not h.value
    assert b"offdiag_sigma" in q.load().qtx_rgf_last_error(None)
    base = q.footprint(q.make_desc(8, 32, "fp64", 4))
    bt = q.footprint(q.make_desc(8, 32, "fp64", 4, offdiag_sigma=True))
    assert bt - base >= 2 * 4 * 32 * 32 * 16
    bt_e = q.footprint(q.make_desc(8, 32, "fp64", 4, offdiag_sigma=True, energy_dependent_sigma=True))
    assert bt_e - bt >= 2 * 7 * 3 * 32 * 32 * 16


def test_fpx_storage_descriptor(libpath):
    """storage_bits must be one of the FPX widths; it replaces the N_B left-connected blocks per kind
    in the sweep's type by two working blocks plus N_B compressed slots, and such plans keep no
    Z_i = V_i g_i and X_i = V_i g^<_i blocks from the forward sweep (2 (N_B - 1) more full blocks
    without FPX storage)."""
    import paper_2606_25595_gb300 as q
    h = ctypes.c_void_p()
    bad = q.make_desc(8, 32, "fp64", 4, storage_bits=33)
    assert q.load().qtx_rgf_plan_create(ctypes.byref(bad), ctypes.byref(h)) == 1 and not h.value
    assert b"storage_bits" in q.load().qtx_rgf_last_error(None)
    nb, b, ec = 64, 256, 16
    base = q.footprint(q.make_desc(nb, b, "emu64", ec))
    for bits in (48, 40, 24):
        fx = q.footprint(q.make_desc(nb, b, "emu64", ec, storage_bits=bits))
        saved = 2 * (nb - 2) * ec * b * b * 16 - 2 * nb * ec * (2 * b * b) * bits // 8 + 2 * (nb - 1) * ec * b * b * 16
        assert abs((base - fx) - saved) < 1 << 20, (bits, base - fx, saved)
    assert q.load().qtx_fpx_bytes(40, 10) == 80


def test_refine_tol_validation(libpath):
    import paper_2606_25595_gb300 as q
    h = ctypes.c_void_p()
    bad = q.make_desc(4, 16, "emu64", 2, refine_tol=-1.0)
    assert q.load().qtx_rgf_plan_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    assert b"refine_tol" in q.load().qtx_rgf_last_error(None)


def test_second_rhs_descriptor(libpath):
    """second_rhs needs system_input and no FPX storage; it keeps one more set of left-connected
    blocks (N_B per energy in flight), one more set of the forward sweep's X_i = V_i g^<_i
    (N_B - 1) and, with block-tridiagonal right-hand sides, one more work block; GG outputs are then
    allowed on a system_input plan."""
    import paper_2606_25595_gb300 as q
    h = ctypes.c_void_p()
    lib = q.load()
    bad = q.make_desc(4, 16, "fp64", 2, second_rhs=True, outputs=["GR_diag"])
    assert lib.qtx_rgf_plan_create(ctypes.byref(bad), ctypes.byref(h)) == 1 and not h.value
    assert b"second_rhs" in lib.qtx_rgf_last_error(None)
    bad = q.make_desc(4, 16, "fp64", 2, system_input=True, second_rhs=True, storage_bits=40,
                      outputs=["GR_diag"])
    assert lib.qtx_rgf_plan_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    assert b"second_rhs" in lib.qtx_rgf_last_error(None)
    nb, b, ec = 8, 32, 4
    kw = dict(energy_dependent_sigma=True, offdiag_sigma=True, system_input=True)
    one = q.footprint(q.make_desc(nb, b, "fp64", ec, outputs=["GR_diag", "GL_diag"], **kw))
    two = q.footprint(q.make_desc(nb, b, "fp64", ec, outputs=["GR_diag", "GL_diag", "GG_diag"],
                                  second_rhs=True, **kw))
    assert two - one == (nb + 1) * ec * b * b * 16 + (nb - 1) * ec * b * b * 16
