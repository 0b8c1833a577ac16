"""Python binding of the GB300 RGF selected-inversion library (``libqtx_rgf.so``, C ABI in
``include/qtx_rgf.h``).

This module only marshals arguments: it builds the ctypes descriptors, hands device pointers
(from torch CUDA tensors) and a CUDA stream to the library, and returns the output tensors.
Every step of the solve runs in the library's CUDA kernels; there is no CPU path.  Importing works
without a GPU (the library loads and its symbols resolve); solving needs one.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["lib", "load", "Desc", "Inputs", "Outputs", "Plan", "Group", "QtxError", "PRECISION",
           "OUT", "solve_device", "solve_w", "WSystem", "footprint", "EXPORTED"]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqtx_rgf.so")

PRECISION = {"fp64": 0, "fp32": 1, "bf16x3": 2, "emu64": 3}
STATUS = {0: "QTX_OK", 1: "QTX_ERR_INVALID_ARG", 2: "QTX_ERR_OOM", 3: "QTX_ERR_CUDA",
          4: "QTX_ERR_SINGULAR", 5: "QTX_ERR_NOT_CONVERGED", 6: "QTX_ERR_TIMEOUT",
          7: "QTX_ERR_UNSUPPORTED"}
OUT = {"GR_diag": 1 << 0, "GR_upper": 1 << 1, "GR_lower": 1 << 2, "GL_diag": 1 << 3,
       "GL_upper": 1 << 4, "GG_diag": 1 << 5, "GG_upper": 1 << 6, "current": 1 << 7,
       "density": 1 << 8, "contact": 1 << 9, "transmission": 1 << 10, "integrals": 1 << 11,
       "continuity": 1 << 12}
BLOCK_OUTPUTS = ("GR_diag", "GR_upper", "GR_lower", "GL_diag", "GL_upper", "GG_diag", "GG_upper")
# Every function the C ABI exports (checked by the CPU tests against include/*.h).
EXPORTED = ("qtx_rgf_plan_create", "qtx_rgf_solve", "qtx_rgf_status", "qtx_rgf_destroy",
            "qtx_rgf_last_error", "qtx_rgf_footprint", "qtx_rgf_version", "qtx_zgemm_batched",
            "qtx_zinv_batched", "qtx_lead_self_energy", "qtx_rgf_set_profiling",
            "qtx_rgf_gemm_profile", "qtx_kernel_launches", "qtx_zgemm_emu64_noalloc",
            "qtx_fpx_bytes", "qtx_fpx_compress", "qtx_fpx_decompress", "qtx_w_assemble",
            "qtx_rgf_group_create", "qtx_rgf_group_solve", "qtx_rgf_group_destroy",
            "qtx_rgf_group_last_error", "qtx_rgf_group_launches", "qtx_rgf_group_pooled_products",
            "qtx_tc_wait_test", "qtx_rgf_group_set_pool_waves")


class QtxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int), ("block_size", ctypes.c_int),
                ("max_energies_in_flight", ctypes.c_int), ("precision", ctypes.c_int),
                ("refine_max_iter", ctypes.c_int), ("has_S", ctypes.c_int),
                ("has_scattering", ctypes.c_int), ("energy_dependent_sigma", ctypes.c_int),
                ("leads", ctypes.c_int), ("decim_tol", ctypes.c_double),
                ("decim_max_iter", ctypes.c_int), ("outputs", ctypes.c_uint),
                ("offdiag_sigma", ctypes.c_int), ("storage_bits", ctypes.c_int),
                ("sigma_stream", ctypes.c_int), ("system_input", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("second_rhs", ctypes.c_int),
                ("escalate_tol", ctypes.c_double), ("tc_stages", ctypes.c_int), ("tc_ctas", ctypes.c_int)]


class Inputs(ctypes.Structure):
    _fields_ = [("H_diag", ctypes.c_void_p), ("H_upper", ctypes.c_void_p),
                ("S_diag", ctypes.c_void_p), ("S_upper", ctypes.c_void_p),
                ("SigR_diag", ctypes.c_void_p), ("SigL_diag", ctypes.c_void_p),
                ("lead_H00_L", ctypes.c_void_p), ("lead_H01_L", ctypes.c_void_p),
                ("lead_H00_R", ctypes.c_void_p), ("lead_H01_R", ctypes.c_void_p),
                ("eta", ctypes.c_double), ("mu_L", ctypes.c_double), ("mu_R", ctypes.c_double),
                ("kT", ctypes.c_double), ("energies", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("n_energies", ctypes.c_int),
                ("n_blocks", ctypes.c_int), ("SigR_upper", ctypes.c_void_p),
                ("SigR_lower", ctypes.c_void_p), ("SigL_upper", ctypes.c_void_p),
                ("M_diag", ctypes.c_void_p), ("M_upper", ctypes.c_void_p), ("M_lower", ctypes.c_void_p),
                ("SigG_diag", ctypes.c_void_p), ("SigG_upper", ctypes.c_void_p)]


class WInputs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("V_diag", "V_upper", "PR_diag", "PR_upper", "PR_lower",
                                               "PL_diag", "PL_upper", "PG_diag", "PG_upper")] + \
               [("n_energies", ctypes.c_int), ("n_blocks", ctypes.c_int)]


class WOutputs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("M_diag", "M_upper", "M_lower", "BL_diag", "BL_upper",
                                               "BG_diag", "BG_upper")]


class Outputs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in BLOCK_OUTPUTS] + \
               [(n, ctypes.c_void_p) for n in ("current", "density", "contact", "transmission",
                                               "current_int", "density_int",
                                               "status_per_energy", "continuity", "escalated")]


_lib = None


def load() -> ctypes.CDLL:
    """Load ``libqtx_rgf.so`` (built in-tree by ``paper_2606_25595_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2606_25595_gb300.build.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    L.qtx_rgf_plan_create.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(ctypes.c_void_p)]
    L.qtx_rgf_plan_create.restype = ctypes.c_int
    L.qtx_rgf_solve.argtypes = [ctypes.c_void_p, ctypes.POINTER(Inputs), ctypes.POINTER(Outputs),
                                ctypes.c_void_p]
    L.qtx_rgf_solve.restype = ctypes.c_int
    L.qtx_rgf_status.argtypes = [ctypes.c_void_p]
    L.qtx_rgf_status.restype = ctypes.c_int
    L.qtx_rgf_destroy.argtypes = [ctypes.c_void_p]
    L.qtx_rgf_destroy.restype = ctypes.c_int
    L.qtx_rgf_last_error.argtypes = [ctypes.c_void_p]
    L.qtx_rgf_last_error.restype = ctypes.c_char_p
    L.qtx_rgf_footprint.argtypes = [ctypes.POINTER(Desc)]
    L.qtx_rgf_footprint.restype = ctypes.c_size_t
    L.qtx_rgf_version.argtypes = []
    L.qtx_rgf_version.restype = ctypes.c_char_p
    vp, i, l, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double
    L.qtx_zgemm_batched.argtypes = [i, i, i, i, i, vp, l, l, i, vp, l, l, d, d, vp, l, l, vp, l, l, i, vp]
    L.qtx_zgemm_batched.restype = i
    L.qtx_zinv_batched.argtypes = [i, i, vp, l, i, i, vp, vp]
    L.qtx_zinv_batched.restype = i
    L.qtx_lead_self_energy.argtypes = [i, vp, vp, vp, i, d, d, i, vp, vp, vp]
    L.qtx_lead_self_energy.restype = i
    L.qtx_rgf_set_profiling.argtypes = [vp, i]
    L.qtx_rgf_set_profiling.restype = i
    L.qtx_rgf_gemm_profile.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(d),
                                       ctypes.POINTER(d), ctypes.POINTER(d)]
    L.qtx_rgf_gemm_profile.restype = i
    L.qtx_kernel_launches.argtypes = []
    L.qtx_kernel_launches.restype = ctypes.c_longlong
    L.qtx_zgemm_emu64_noalloc.argtypes = [i, i, i, i, vp, l, l, i, vp, l, l, d, d, vp, l, l, vp, l, l, i, vp]
    L.qtx_zgemm_emu64_noalloc.restype = i
    L.qtx_w_assemble.argtypes = [ctypes.c_void_p, ctypes.POINTER(WInputs), ctypes.POINTER(WOutputs), vp]
    L.qtx_w_assemble.restype = i
    L.qtx_rgf_group_create.argtypes = [i, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p)]
    L.qtx_rgf_group_create.restype = i
    L.qtx_rgf_group_solve.argtypes = [vp, ctypes.POINTER(ctypes.POINTER(Inputs)), ctypes.POINTER(ctypes.POINTER(Outputs)), vp]
    L.qtx_rgf_group_solve.restype = i
    L.qtx_rgf_group_destroy.argtypes = [vp]
    L.qtx_rgf_group_destroy.restype = i
    L.qtx_rgf_group_last_error.argtypes = [vp]
    L.qtx_rgf_group_last_error.restype = ctypes.c_char_p
    L.qtx_rgf_group_launches.argtypes = [vp]
    L.qtx_rgf_group_launches.restype = ctypes.c_longlong
    L.qtx_rgf_group_set_pool_waves.argtypes = [vp, i]
    L.qtx_rgf_group_set_pool_waves.restype = i
    L.qtx_rgf_group_pooled_products.argtypes = [vp]
    L.qtx_rgf_group_pooled_products.restype = ctypes.c_longlong
    L.qtx_tc_wait_test.argtypes = [i]
    L.qtx_tc_wait_test.restype = i
    L.qtx_fpx_bytes.argtypes = [i, l]
    L.qtx_fpx_bytes.restype = ctypes.c_size_t
    L.qtx_fpx_compress.argtypes = [i, vp, l, d, vp, vp]
    L.qtx_fpx_compress.restype = i
    L.qtx_fpx_decompress.argtypes = [i, vp, l, vp, vp]
    L.qtx_fpx_decompress.restype = i
    _lib = L
    return L


def lib() -> ctypes.CDLL:
    return load()


def make_desc(n_blocks, block_size, precision="fp64", max_energies_in_flight=64,
              refine_max_iter=2, has_S=False, has_scattering=True, energy_dependent_sigma=False,
              leads=False, decim_tol=1e-13, decim_max_iter=100, outputs=None,
              offdiag_sigma=False, storage_bits=0, sigma_stream=False, system_input=False,
              refine_tol=0.0, second_rhs=False, escalate_tol=0.0, tc_stages=0, tc_ctas=0) -> Desc:
    if outputs is None:
        outputs = (1 << 12) - 1  # every output but the continuity residual
    elif not isinstance(outputs, int):
        mask = 0
        for name in outputs:
            mask |= OUT[name]
        outputs = mask
    return Desc(int(n_blocks), int(block_size), int(max_energies_in_flight),
                PRECISION[precision] if isinstance(precision, str) else int(precision),
                int(refine_max_iter), int(bool(has_S)), int(bool(has_scattering)),
                int(bool(energy_dependent_sigma)), int(bool(leads)), float(decim_tol),
                int(decim_max_iter), int(outputs), int(bool(offdiag_sigma)), int(storage_bits),
                int(bool(sigma_stream)), int(bool(system_input)), float(refine_tol),
                int(bool(second_rhs)), float(escalate_tol), int(tc_stages), int(tc_ctas))


def kernel_launches() -> int:
    return int(load().qtx_kernel_launches())


def footprint(desc: Desc) -> int:
    return int(load().qtx_rgf_footprint(ctypes.byref(desc)))


class Plan:
    """Owns a ``qtx_rgf_plan`` (device workspace for one shape / precision)."""

    def __init__(self, desc: Desc):
        L = load()
        self.desc = desc
        h = ctypes.c_void_p()
        s = L.qtx_rgf_plan_create(ctypes.byref(desc), ctypes.byref(h))
        if s != 0:
            raise QtxError(s, L.qtx_rgf_last_error(None).decode())
        self._h = h

    def _check(self, s):
        if s != 0:
            raise QtxError(s, load().qtx_rgf_last_error(self._h).decode())

    def solve(self, inputs: Inputs, outputs: Outputs, stream: int = 0) -> None:
        self._check(load().qtx_rgf_solve(self._h, ctypes.byref(inputs), ctypes.byref(outputs),
                                         ctypes.c_void_p(stream)))

    def w_assemble(self, inputs: "WInputs", outputs: "WOutputs", stream: int = 0) -> None:
        self._check(load().qtx_w_assemble(self._h, ctypes.byref(inputs), ctypes.byref(outputs),
                                          ctypes.c_void_p(stream)))

    def status(self) -> int:
        return int(load().qtx_rgf_status(self._h))

    def set_profiling(self, on: bool = True) -> None:
        self._check(load().qtx_rgf_set_profiling(self._h, int(bool(on))))

    def gemm_profile(self) -> dict:
        n, ms, pf, uf = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(load().qtx_rgf_gemm_profile(self._h, ctypes.byref(n), ctypes.byref(ms),
                                                ctypes.byref(pf), ctypes.byref(uf)))
        return dict(launches=n.value, ms=ms.value, pipe_flops=pf.value, useful_flops=uf.value)

    def close(self):
        if getattr(self, "_h", None):
            load().qtx_rgf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Owns a ``qtx_rgf_group``: several plans solved together, their tensor-core products pooled
    into shared persistent launches (include/qtx_rgf.h).  Marshalling only."""

    def __init__(self, plans: list):
        L = load()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(plans))(*[p._h for p in plans])
        h = ctypes.c_void_p()
        s = L.qtx_rgf_group_create(len(plans), arr, ctypes.byref(h))
        if s != 0:
            raise QtxError(s, L.qtx_rgf_group_last_error(None).decode())
        self._h = h

    def solve(self, inputs: list, outputs: list, stream: int = 0) -> None:
        L = load()
        ia = (ctypes.POINTER(Inputs) * len(inputs))(*[ctypes.pointer(x) for x in inputs])
        oa = (ctypes.POINTER(Outputs) * len(outputs))(*[ctypes.pointer(x) for x in outputs])
        s = L.qtx_rgf_group_solve(self._h, ia, oa, ctypes.c_void_p(stream))
        if s != 0:
            raise QtxError(s, L.qtx_rgf_group_last_error(self._h).decode())

    def set_pool_waves(self, waves: int) -> None:
        s = load().qtx_rgf_group_set_pool_waves(self._h, int(waves))
        if s != 0:
            raise QtxError(s, "qtx_rgf_group_set_pool_waves")

    def launches(self) -> int:
        return int(load().qtx_rgf_group_launches(self._h))

    def pooled_products(self) -> int:
        return int(load().qtx_rgf_group_pooled_products(self._h))

    def close(self):
        if getattr(self, "_h", None):
            load().qtx_rgf_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class WSystem:
    """Screened-Coulomb system (Table I, W row) resident on the GPU: the inputs of a
    ``workloads.w_system`` dict uploaded once, a system_input plan, and the assembled and solved
    blocks.  ``run()`` assembles M = I - V P^R and B^<> = V P^<> V^H (BT blocks, ``qtx_w_assemble``)
    and solves M X M^H = B for X^R (BT blocks of M^-1) and X^< from B^<, and X^> from B^> as the
    plan's second right-hand side, in one solve that shares the retarded sweep.  Marshalling only."""

    def __init__(self, w: dict, precision: str = "emu64", max_energies_in_flight=64, greater=True):
        import torch
        cd = torch.device("cuda")
        nb, b, ne = w["n_blocks"], w["block_size"], w["n_energies"]
        self.nb, self.b, self.ne, self.greater = nb, b, ne, greater
        nu = max(nb - 1, 0)

        def T(x):
            return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.complex128).to(cd)

        def E(*shape):
            return torch.empty(shape, dtype=torch.complex128, device=cd)

        self.win, self.wout, self._keep = WInputs(), WOutputs(), {}
        for k in ("V_diag", "V_upper", "PR_diag", "PR_upper", "PR_lower", "PL_diag", "PL_upper") + \
                (("PG_diag", "PG_upper") if greater else ()):
            self._keep[k] = T(w[k])
            setattr(self.win, k, self._keep[k].data_ptr() if self._keep[k].numel() else None)
        self.win.n_energies, self.win.n_blocks = ne, nb
        self.res = {"M_diag": E(ne, nb, b, b), "M_upper": E(ne, nu, b, b), "M_lower": E(ne, nu, b, b),
                    "BL_diag": E(ne, nb, b, b), "BL_upper": E(ne, nu, b, b)}
        if greater:
            self.res.update(BG_diag=E(ne, nb, b, b), BG_upper=E(ne, nu, b, b))
        for k, v in self.res.items():
            setattr(self.wout, k, v.data_ptr() if v.numel() else None)
        outs = ["GR_diag", "GR_upper", "GR_lower", "GL_diag", "GL_upper"] + \
            (["GG_diag", "GG_upper"] if greater else [])
        self.plan = Plan(make_desc(nb, b, precision, min(max_energies_in_flight, ne), 2, has_scattering=True,
                                   energy_dependent_sigma=True, offdiag_sigma=nb > 1, system_input=True,
                                   outputs=outs, second_rhs=greater))
        self.energies = torch.zeros(ne, dtype=torch.float64, device=cd)
        self.res["status"] = torch.zeros(ne, dtype=torch.int32, device=cd)
        keys = [("GR_diag", "XR_diag"), ("GR_upper", "XR_upper"), ("GR_lower", "XR_lower"),
                ("GL_diag", "XL_diag"), ("GL_upper", "XL_upper")]
        if greater:
            keys += [("GG_diag", "XG_diag"), ("GG_upper", "XG_upper")]
        inp = Inputs()
        inp.M_diag = self.res["M_diag"].data_ptr()
        inp.M_upper = self.res["M_upper"].data_ptr() if nu else None
        inp.M_lower = self.res["M_lower"].data_ptr() if nu else None
        inp.SigL_diag = self.res["BL_diag"].data_ptr()
        inp.SigL_upper = self.res["BL_upper"].data_ptr() if nu else None
        if greater:
            inp.SigG_diag = self.res["BG_diag"].data_ptr()
            inp.SigG_upper = self.res["BG_upper"].data_ptr() if nu else None
        inp.energies, inp.n_energies, inp.n_blocks = self.energies.data_ptr(), ne, nb
        o = Outputs()
        for name, key in keys:
            self.res[key] = E(ne, nb if "diag" in name else nu, b, b)
            setattr(o, name, self.res[key].data_ptr() if self.res[key].numel() else None)
        o.status_per_energy = self.res["status"].data_ptr()
        self._solve = (inp, o)

    def run(self, stream=None):
        st = _stream(stream)
        self.plan.w_assemble(self.win, self.wout, st)
        self.plan.solve(*self._solve, st)

    def results(self) -> dict:
        import torch
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in self.res.items()}

    def close(self):
        self.plan.close()


def solve_w(w: dict, precision: str = "emu64", max_energies_in_flight=64, greater=True, stream=None):
    """One-shot ``WSystem``: upload, assemble, solve, return numpy arrays (M_*, BL_*, BG_*, XR_*,
    XL_*, XG_*, status)."""
    ws = WSystem(w, precision, max_energies_in_flight, greater)
    ws.run(stream)
    out = ws.results()
    ws.close()
    return out


def has_offdiag_sigma(dev: dict) -> bool:
    """True when a device dict carries block-tridiagonal scattering self-energies."""
    return any(dev.get(k) is not None for k in ("SigR_upper", "SigR_lower", "SigL_upper"))


def solve_device(dev: dict, precision: str = "fp64", outputs=None, max_energies_in_flight=64,
                 refine_max_iter=2, weights=None, energies=None, stream=None, plan=None,
                 device_inputs=None, keep_on_device=False, storage_bits=0, sigma_stream=False,
                 escalate_tol=0.0):
    """Solve a ``workloads``-style device dict on the GPU and return numpy arrays (or tensors).

    Marshalling only: inputs are copied to torch CUDA tensors (complex128), the C ABI is called on
    the current torch stream, and the requested outputs come back.  ``device_inputs`` reuses
    already-uploaded tensors (see ``upload``).
    """
    import torch

    nb, b = dev["n_blocks"], dev["block_size"]
    E = np.asarray(dev["energies"] if energies is None else energies, dtype=np.float64)
    ne = E.size
    din = device_inputs if device_inputs is not None else upload(dev, E, weights, sigma_host=sigma_stream)
    want = list(outputs) if outputs is not None else [k for k in OUT if k != "continuity"]
    if not dev.get("leads"):
        want = [w for w in want if w not in ("contact", "transmission")]
    desc = make_desc(nb, b, precision, min(max_energies_in_flight, ne), refine_max_iter,
                     has_S=dev.get("S_diag") is not None, has_scattering=dev.get("SigR") is not None,
                     energy_dependent_sigma=dev.get("SigR") is not None and dev["SigR"].shape[0] > 1,
                     leads=bool(dev.get("leads")), outputs=want, offdiag_sigma=has_offdiag_sigma(dev),
                     storage_bits=storage_bits, sigma_stream=sigma_stream, escalate_tol=escalate_tol)
    P = plan if plan is not None else Plan(desc)
    cdev = torch.device("cuda")
    res = {}
    shapes = {"GR_diag": (ne, nb, b, b), "GR_upper": (ne, nb - 1, b, b),
              "GR_lower": (ne, nb - 1, b, b), "GL_diag": (ne, nb, b, b),
              "GL_upper": (ne, nb - 1, b, b), "GG_diag": (ne, nb, b, b),
              "GG_upper": (ne, nb - 1, b, b), "current": (ne, nb - 1), "density": (ne, nb),
              "contact": (ne, 2), "transmission": (ne,), "integrals": None, "continuity": (ne,)}
    o = Outputs()
    for k in want:
        if k == "integrals":
            res["current_int"] = torch.zeros(max(nb - 1, 0), dtype=torch.float64, device=cdev)
            res["density_int"] = torch.zeros(nb, dtype=torch.float64, device=cdev)
            o.current_int = res["current_int"].data_ptr() if nb > 1 else None
            o.density_int = res["density_int"].data_ptr()
            continue
        shp = shapes[k]
        if 0 in shp:
            continue
        dt = torch.complex128 if k in BLOCK_OUTPUTS else torch.float64
        res[k] = torch.empty(shp, dtype=dt, device=cdev)
        setattr(o, k, res[k].data_ptr())
    res["status"] = torch.zeros(ne, dtype=torch.int32, device=cdev)
    o.status_per_energy = res["status"].data_ptr()
    if escalate_tol > 0:
        res["escalated"] = torch.zeros(ne, dtype=torch.int32, device=cdev)
        o.escalated = res["escalated"].data_ptr()
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    P.solve(din["_inputs"], o, st)
    torch.cuda.current_stream().synchronize()
    if keep_on_device:
        return res
    return {k: v.cpu().numpy() for k, v in res.items()}


def upload(dev: dict, energies=None, weights=None, sigma_host=False) -> dict:
    """Copy a device dict's blocks to torch CUDA tensors and build the ``Inputs`` struct.

    ``sigma_host``: keep the (energy-dependent) scattering self-energies in pinned host memory for a
    plan with ``sigma_stream``."""
    import torch

    cdev = torch.device("cuda")

    def T(x, dt=torch.complex128):
        return None if x is None else torch.as_tensor(np.ascontiguousarray(x), dtype=dt).to(cdev)

    def Th(x):
        return None if x is None else torch.as_tensor(np.ascontiguousarray(x), dtype=torch.complex128).pin_memory()

    E = np.asarray(dev["energies"] if energies is None else energies, dtype=np.float64)
    d = {"H_diag": T(dev["H_diag"]), "H_upper": T(dev["H_upper"]) if dev["n_blocks"] > 1 else None,
         "S_diag": T(dev.get("S_diag")), "S_upper": T(dev.get("S_upper")),
         "SigR_diag": None, "SigL_diag": None, "energies": T(E, torch.float64),
         "weights": T(weights, torch.float64) if weights is not None else None}
    if dev.get("SigR") is not None:
        SR, SL = dev["SigR"], dev["SigL"]
        put = Th if sigma_host else T
        d["SigR_diag"] = put(SR[0] if SR.shape[0] == 1 else SR)
        d["SigL_diag"] = put(SL[0] if SL.shape[0] == 1 else SL)
    for k in ("SigR_upper", "SigR_lower", "SigL_upper"):
        X = dev.get(k)
        d[k] = None if X is None or X.size == 0 else T(X[0] if X.shape[0] == 1 else X)
    leads = dev.get("leads") or {}
    for k in ("H00_L", "H01_L", "H00_R", "H01_R"):
        d["lead_" + k] = T(leads.get(k))
    inp = Inputs()
    for k in ("H_diag", "H_upper", "S_diag", "S_upper", "SigR_diag", "SigL_diag", "lead_H00_L",
              "lead_H01_L", "lead_H00_R", "lead_H01_R", "energies", "weights", "SigR_upper",
              "SigR_lower", "SigL_upper"):
        setattr(inp, k, None if d[k] is None else d[k].data_ptr())
    inp.eta = float(dev["eta"])
    inp.mu_L = float(dev.get("mu_L", 0.0))
    inp.mu_R = float(dev.get("mu_R", 0.0))
    inp.kT = float(dev.get("kT", 0.025))
    inp.n_energies = int(E.size)
    d["_inputs"] = inp
    return d


def _stream(stream):
    import torch
    return torch.cuda.current_stream().cuda_stream if stream is None else stream


def zgemm_batched(A, B, precision="emu64", opA="N", opB="N", alpha=1.0, beta=0.0, C0=None,
                  stream=None):
    """C[e] = alpha op(A[e]) op(B[e]) + beta C0[e] on complex128 CUDA tensors [batch, rows, cols]
    (a 2-D tensor is shared by the whole batch).  Marshalling only; the product runs in the
    library's kernels."""
    import torch
    ops = {"N": 0, "C": 1}
    A3 = A if A.dim() == 3 else A.unsqueeze(0)
    B3 = B if B.dim() == 3 else B.unsqueeze(0)
    batch = max(A3.shape[0] if A.dim() == 3 else 1, B3.shape[0] if B.dim() == 3 else 1)
    M = A3.shape[1] if opA == "N" else A3.shape[2]
    K = A3.shape[2] if opA == "N" else A3.shape[1]
    N = B3.shape[2] if opB == "N" else B3.shape[1]
    C = torch.empty((batch, M, N), dtype=torch.complex128, device=A.device)
    c0p, ldc0, sc0 = None, N, 0
    if C0 is not None:
        C03 = C0 if C0.dim() == 3 else C0.unsqueeze(0)
        c0p, ldc0, sc0 = C03.data_ptr(), C03.shape[2], (C03.shape[1] * C03.shape[2] if C0.dim() == 3 else 0)
    s = load().qtx_zgemm_batched(
        PRECISION[precision], M, N, K, ops[opA], A3.data_ptr(), A3.shape[2],
        A3.shape[1] * A3.shape[2] if A.dim() == 3 else 0, ops[opB], B3.data_ptr(), B3.shape[2],
        B3.shape[1] * B3.shape[2] if B.dim() == 3 else 0, float(alpha), float(beta), c0p, ldc0, sc0,
        C.data_ptr(), N, M * N, batch, ctypes.c_void_p(_stream(stream)))
    if s != 0:
        raise QtxError(s, "qtx_zgemm_batched")
    return C


def fpx_compress(x, bits, cutoff=0.0, stream=None):
    """FPX codes (uint8 CUDA tensor of qtx_fpx_bytes(bits, n) bytes) of a float64 or complex128 CUDA
    tensor's n real values.  Marshalling only; the rounding runs in the library's kernel."""
    import torch
    xr = torch.view_as_real(x) if x.is_complex() else x
    xr = xr.contiguous()
    n = xr.numel()
    out = torch.empty(max(int(load().qtx_fpx_bytes(int(bits), n)), 8), dtype=torch.uint8, device=x.device)
    s = load().qtx_fpx_compress(int(bits), xr.data_ptr(), n, float(cutoff), out.data_ptr(),
                                ctypes.c_void_p(_stream(stream)))
    if s != 0:
        raise QtxError(s, "qtx_fpx_compress")
    return out


def fpx_decompress(codes, bits, n, complex_out=False, stream=None):
    """n FP64 values (n/2 complex128 values if ``complex_out``) decoded from FPX codes."""
    import torch
    x = torch.empty(n, dtype=torch.float64, device=codes.device)
    s = load().qtx_fpx_decompress(int(bits), codes.data_ptr(), int(n), x.data_ptr(),
                                  ctypes.c_void_p(_stream(stream)))
    if s != 0:
        raise QtxError(s, "qtx_fpx_decompress")
    return torch.view_as_complex(x.view(-1, 2)) if complex_out else x


def zinv_batched(A, precision="fp64", refine_iter=2, stream=None):
    """In-place batched inverse of complex128 CUDA tensor A [batch, n, n]; returns (A, status)."""
    import torch
    status = torch.zeros(A.shape[0], dtype=torch.int32, device=A.device)
    s = load().qtx_zinv_batched(PRECISION[precision], A.shape[1], A.data_ptr(), A.shape[1] * A.shape[2],
                                A.shape[0], int(refine_iter), status.data_ptr(),
                                ctypes.c_void_p(_stream(stream)))
    if s != 0:
        raise QtxError(s, "qtx_zinv_batched")
    return A, status


def lead_self_energy(H00, H01, energies, eta, tol=1e-13, max_iter=100, stream=None):
    """Contact Sigma^R(E) [n_E, n, n] from CUDA tensors H00, H01 (complex128) and energies (float64)."""
    import torch
    n = H00.shape[0]
    out = torch.empty((energies.shape[0], n, n), dtype=torch.complex128, device=H00.device)
    status = torch.zeros(energies.shape[0], dtype=torch.int32, device=H00.device)
    s = load().qtx_lead_self_energy(n, H00.data_ptr(), H01.data_ptr(), energies.data_ptr(),
                                    energies.shape[0], float(eta), float(tol), int(max_iter),
                                    out.data_ptr(), status.data_ptr(), ctypes.c_void_p(_stream(stream)))
    if s != 0:
        raise QtxError(s, "qtx_lead_self_energy")
    return out, status
