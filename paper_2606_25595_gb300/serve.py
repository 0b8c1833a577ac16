"""Continuous-batching request loop for RGF solves on one GPU (host-side scheduling only; every solve
runs in the library's kernels through the C ABI).

* Device models (H, Sigma blocks of a device) stay resident in HBM; a request is an energy-sweep /
  bias-point solve on the first ``n_blocks`` slices of one model, with its own energy grid, contact
  chemical potentials and precision.
* Plans (device workspaces) are pooled per (block size, precision) and sized for the model's full
  length; a pool grows only when its HBM footprint (``qtx_rgf_footprint``) fits the budget.
* Each of ``slots`` CUDA streams runs one request at a time; requests that arrive while others are on
  the GPU are admitted as soon as a slot, a plan and memory are free, so their work overlaps on the
  device.  Completion is detected by polling CUDA events; latency = completion - arrival.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import Inputs, Outputs, Plan, footprint, make_desc

__all__ = ["DeviceModel", "Request", "Server"]


class DeviceModel:
    """Device blocks resident on the GPU (complex128), usable by prefix of ``n_blocks`` slices."""

    def __init__(self, dev: dict, key: str):
        import torch
        cd = torch.device("cuda")

        def T(x):
            return None if x is None else torch.as_tensor(np.ascontiguousarray(x), dtype=torch.complex128).to(cd)

        self.key = key
        self.b = dev["block_size"]
        self.n_blocks = dev["n_blocks"]
        self.eta = float(dev["eta"])
        self.H_diag = T(dev["H_diag"])
        self.H_upper = T(dev["H_upper"])
        self.SigR = T(dev["SigR"][0]) if dev.get("SigR") is not None else None
        self.SigL = T(dev["SigL"][0]) if dev.get("SigL") is not None else None


@dataclass
class Request:
    rid: int
    model: str
    n_blocks: int
    energies: np.ndarray
    precision: str = "emu64"
    mu_L: float = 0.0
    mu_R: float = 0.0
    t_arrival: float = 0.0
    # filled by the server
    t_start: float = -1.0
    t_done: float = -1.0
    result: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class Server:
    """Admit requests as they arrive and overlap their solves on ``slots`` CUDA streams."""

    def __init__(self, models: dict, slots: int = 4, hbm_budget: int | None = None,
                 chunk_by_b: dict | None = None, refine_max_iter: int = 2):
        import torch
        self.models = models
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.busy: list = [None] * slots  # (request, plan, event, buffers)
        free, _ = torch.cuda.mem_get_info()
        self.budget = hbm_budget if hbm_budget is not None else int(free * 0.6)
        self.used = 0
        self.pools: dict = {}             # (b, nb_max, precision) -> list of idle plans
        self.chunk_by_b = chunk_by_b or {64: 128, 128: 64, 256: 32, 512: 16, 1024: 8}
        self.refine = refine_max_iter
        self.queue: list = []
        self.done: list = []

    # ------------------------------------------------------------------ plans
    def _desc(self, m: DeviceModel, precision: str, n_e: int):
        ec = min(self.chunk_by_b.get(m.b, 16), n_e)
        return make_desc(m.n_blocks, m.b, precision, ec, self.refine, has_scattering=m.SigR is not None,
                         outputs=["current", "density", "integrals"])

    def _take_plan(self, m: DeviceModel, precision: str):
        key = (m.b, m.n_blocks, precision)
        pool = self.pools.setdefault(key, [])
        if pool:
            return pool.pop()
        d = self._desc(m, precision, 1 << 30)
        need = footprint(d)
        if self.used + need > self.budget:
            return None
        p = Plan(d)
        p.key, p.bytes = key, need
        self.used += need
        return p

    def warm(self, precisions=("emu64", "fp32"), per_key: int = 1):
        """Create plans ahead of time (plan creation allocates and would stall the loop)."""
        for m in self.models.values():
            for prec in precisions:
                plans = [self._take_plan(m, prec) for _ in range(per_key)]
                for p in plans:
                    if p is not None:
                        self.pools[p.key].append(p)

    # ------------------------------------------------------------------ request lifecycle
    def submit(self, req: Request):
        self.queue.append(req)

    def _start(self, slot: int, req: Request, plan: Plan):
        import torch
        m = self.models[req.model]
        nb, ne = req.n_blocks, len(req.energies)
        st = self.streams[slot]
        with torch.cuda.stream(st):
            E = torch.as_tensor(req.energies, dtype=torch.float64).cuda(non_blocking=False)
            cur = torch.empty((ne, max(nb - 1, 1)), dtype=torch.float64, device="cuda")
            den = torch.empty((ne, nb), dtype=torch.float64, device="cuda")
            cint = torch.zeros(max(nb - 1, 1), dtype=torch.float64, device="cuda")
            dint = torch.zeros(nb, dtype=torch.float64, device="cuda")
            stat = torch.zeros(ne, dtype=torch.int32, device="cuda")
        inp = Inputs()
        inp.H_diag = m.H_diag.data_ptr()
        inp.H_upper = m.H_upper.data_ptr()
        inp.SigR_diag = m.SigR.data_ptr() if m.SigR is not None else None
        inp.SigL_diag = m.SigL.data_ptr() if m.SigL is not None else None
        inp.eta, inp.mu_L, inp.mu_R, inp.kT = m.eta, req.mu_L, req.mu_R, 0.025
        inp.energies = E.data_ptr()
        inp.n_energies = ne
        inp.n_blocks = nb
        out = Outputs()
        out.current = cur.data_ptr() if nb > 1 else None
        out.density = den.data_ptr()
        out.current_int = cint.data_ptr() if nb > 1 else None
        out.density_int = dint.data_ptr()
        out.status_per_energy = stat.data_ptr()
        plan.solve(inp, out, st.cuda_stream)
        ev = torch.cuda.Event()
        ev.record(st)
        req.t_start = time.perf_counter()
        self.busy[slot] = (req, plan, ev, (E, cur, den, cint, dint, stat))

    def _finish(self, slot: int):
        req, plan, ev, (E, cur, den, cint, dint, stat) = self.busy[slot]
        req.t_done = time.perf_counter()
        req.result = {"current": cur.cpu().numpy() if req.n_blocks > 1 else np.zeros((len(req.energies), 0)),
                      "density": den.cpu().numpy(), "current_int": cint.cpu().numpy(),
                      "density_int": dint.cpu().numpy(), "status": stat.cpu().numpy()}
        self.pools[plan.key].append(plan)
        self.busy[slot] = None
        self.done.append(req)

    def poll(self) -> bool:
        """Retire finished requests and admit queued ones; returns True if anything changed."""
        changed = False
        for s, item in enumerate(self.busy):
            if item is not None and item[2].query():
                self._finish(s)
                changed = True
        for s in range(len(self.busy)):
            if self.busy[s] is not None or not self.queue:
                continue
            # FIFO with skip-ahead: the first queued request whose plan is available or fits
            for qi, req in enumerate(self.queue):
                plan = self._take_plan(self.models[req.model], req.precision)
                if plan is not None:
                    self.queue.pop(qi)
                    self._start(s, req, plan)
                    changed = True
                    break
        return changed

    def run(self, requests: list, time_limit: float = 600.0) -> dict:
        """Replay ``requests`` (their ``t_arrival`` are offsets in seconds from now) to completion."""
        pending = sorted(requests, key=lambda r: r.t_arrival)
        t0 = time.perf_counter()
        i = 0
        while i < len(pending) or self.queue or any(x is not None for x in self.busy):
            now = time.perf_counter() - t0
            if now > time_limit:
                break
            while i < len(pending) and pending[i].t_arrival <= now:
                pending[i].t_arrival = t0 + pending[i].t_arrival
                self.submit(pending[i])
                i += 1
            if not self.poll():
                time.sleep(0.0002)
        t1 = time.perf_counter()
        done = [r for r in self.done if r in requests]
        lat = np.array([r.latency for r in done]) if done else np.zeros(0)
        pts = sum(len(r.energies) for r in done)
        return {"completed": len(done), "submitted": len(requests), "wall_s": t1 - t0,
                "energy_points_per_s": pts / (t1 - t0) if t1 > t0 else 0.0,
                "requests_per_s": len(done) / (t1 - t0) if t1 > t0 else 0.0,
                "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                "hbm_plans_bytes": int(self.used)}
