"""Continuous-batching request loop for RGF solves on one GPU (host-side scheduling only; every solve
runs in the library's kernels through the C ABI).

* Device models (H, Sigma blocks of a device) stay resident in HBM; a request is an energy-sweep /
  bias-point solve on the first ``n_blocks`` slices of one model, with its own energy grid, contact
  chemical potentials and precision.
* Plans (device workspaces) are pooled per (block size, precision) and sized for the model's full
  length (``PlanPool``); a pool grows only when its HBM footprint (``qtx_rgf_footprint``) fits the
  budget, and when it does not, idle plans of other keys are closed to make room, so that a request
  whose plan fits the budget alone is always admitted once the batches ahead of it finish.  A request
  whose plan could never fit the budget is refused when it is submitted (its result says why).
* Each of ``slots`` CUDA streams runs one batch at a time: the queued requests admitted together
  (up to ``group_size``, each with a plan of its own) are solved as one ``qtx_rgf_group``: each
  request's solve is enqueued from its own host thread onto its own stream, so their launches overlap
  on the device, while every request keeps its own outputs -- results equal to solving it alone, bit
  for bit.  Requests that arrive while others are on
  the GPU are admitted as soon as a slot, plans and memory are free, so their work overlaps on the
  device.  Completion is detected by polling CUDA events; latency = completion - arrival.
"""
from __future__ import annotations

import functools
import time
from dataclasses import dataclass, field

import numpy as np

from . import Group, Inputs, Outputs, Plan, footprint, make_desc

__all__ = ["DeviceModel", "PlanPool", "Request", "Server"]


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


class PlanPool:
    """Idle plans per key within an HBM budget (host bookkeeping only; ``create(key)`` makes a plan,
    whose ``close()`` frees its workspace).

    ``take`` hands out an idle plan of the key, else creates one if ``used + need`` fits the budget.
    Failing both, a key that has plans in use waits for one of them to come back (None), while a key
    with no plan at all first closes idle plans of other keys (the largest first) until its plan fits.
    Plans in use are never closed, so a key without plans waits only while the plans in use hold too
    much of the budget; once they are given back it is served for any ``need`` <= budget.  Without
    the eviction step a key that found the budget filled by other keys' idle plans would wait for
    ever; evicting only for keys without plans keeps the device synchronisation of a close off the
    common path."""

    def __init__(self, budget: int, create):
        self.budget = int(budget)
        self.create = create
        self.used = 0
        self.idle: dict = {}              # key -> list of (plan, bytes)
        self.size: dict = {}              # id(plan) -> (key, bytes) of every plan the pool made
        self.count: dict = {}             # key -> plans of the key, idle or in use
        self.evicted = 0

    def _evict_for(self, key, need: int) -> bool:
        while self.used + need > self.budget:
            victims = [(b, k) for k, lst in self.idle.items() if k != key for _, b in lst]
            if not victims:
                return False
            b, k = max(victims, key=lambda v: v[0])
            lst = self.idle[k]
            i = next(j for j, (_, bj) in enumerate(lst) if bj == b)
            plan, _ = lst.pop(i)
            self._drop(plan, k, b)
            self.evicted += 1
        return True

    def _make(self, key, need: int):
        plan = self.create(key)
        self.size[id(plan)] = (key, int(need))
        self.count[key] = self.count.get(key, 0) + 1
        self.used += int(need)
        return plan

    def _drop(self, plan, key, b: int):
        del self.size[id(plan)]
        self.count[key] -= 1
        plan.close()
        self.used -= b

    def take(self, key, need: int):
        lst = self.idle.setdefault(key, [])
        if lst:
            return lst.pop()[0]
        if need > self.budget:
            return None
        if self.used + need > self.budget and (self.count.get(key, 0) or not self._evict_for(key, need)):
            return None
        return self._make(key, need)

    def give(self, plan):
        key, b = self.size[id(plan)]
        self.idle.setdefault(key, []).append((plan, b))

    def warm(self, wanted: list, per_key: int = 1):
        """Create up to ``per_key`` idle plans for each (key, need) of ``wanted``, one round over all
        keys at a time, so that every key gets a plan before any key gets a second; never evicts."""
        for r in range(per_key):
            for key, need in wanted:
                lst = self.idle.setdefault(key, [])
                if len(lst) <= r and self.used + need <= self.budget:
                    lst.append((self._make(key, need), int(need)))

    def close(self):
        """Close the idle plans (plans still handed out stay open and counted)."""
        for key, lst in self.idle.items():
            for plan, b in lst:
                self._drop(plan, key, b)
        self.idle.clear()


def _serving_desc(key, chunk_by_b: dict, refine: int):
    b, nb, scat, precision = key
    return make_desc(nb, b, precision, chunk_by_b.get(b, 16), refine, has_scattering=scat,
                     outputs=["current", "density", "integrals"])


def _new_plan(key, chunk_by_b: dict, refine: int):
    p = Plan(_serving_desc(key, chunk_by_b, refine))
    p.key = key
    return p


class Server:
    """Admit requests as they arrive and overlap their solves on ``slots`` CUDA streams."""

    def __init__(self, models: dict, slots: int = 4, hbm_budget: int | None = None,
                 chunk_by_b: dict | None = None, refine_max_iter: int = 2, group_size: int = 4):
        import torch
        self.models = models
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.busy: list = [None] * slots  # (batch of (request, plan, buffers), group, event)
        self.group_size = max(1, min(int(group_size), 8))
        self.rejected: list = []
        self.batches = 0
        self.largest_batch = 0
        free, _ = torch.cuda.mem_get_info()
        self.budget = hbm_budget if hbm_budget is not None else int(free * 0.6)
        self.chunk_by_b = dict(chunk_by_b or {64: 128, 128: 64, 256: 32, 512: 16, 1024: 8})
        self.refine = refine_max_iter
        # keys (b, nb_max, scattering, precision); the factory holds no reference to the server, so
        # the plans are freed as soon as the server is dropped
        self.plans = PlanPool(self.budget, functools.partial(_new_plan, chunk_by_b=self.chunk_by_b,
                                                             refine=self.refine))
        self.queue: list = []
        self.done: list = []

    # ------------------------------------------------------------------ plans
    def _key(self, m: DeviceModel, precision: str):
        return (m.b, m.n_blocks, m.SigR is not None, precision)

    def _desc(self, key):
        return _serving_desc(key, self.chunk_by_b, self.refine)

    def _take_plan(self, m: DeviceModel, precision: str):
        key = self._key(m, precision)
        return self.plans.take(key, footprint(self._desc(key)))

    def warm(self, precisions=("emu64", "fp32"), per_key: int = 1):
        """Create plans ahead of time (plan creation allocates and would stall the loop): up to
        ``per_key`` per (model, precision), every key served once before any key twice."""
        keys = dict.fromkeys(self._key(m, prec) for m in self.models.values() for prec in precisions)
        wanted = [(k, footprint(self._desc(k))) for k in keys]
        self.plans.warm(wanted, per_key)

    # ------------------------------------------------------------------ request lifecycle
    def submit(self, req: Request):
        """Queue a request, or refuse it at once when its plan could never fit the HBM budget."""
        m = self.models[req.model]
        need = footprint(self._desc(self._key(m, req.precision)))
        if need > self.budget:
            req.result = {"rejected": f"plan footprint {need} bytes exceeds the HBM budget {self.budget}"}
            req.t_done = time.perf_counter()
            self.rejected.append(req)
            return
        self.queue.append(req)

    def _buffers(self, req: Request, plan: Plan):
        import torch
        m = self.models[req.model]
        nb, ne = req.n_blocks, len(req.energies)
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
        return inp, out, (E, cur, den, cint, dint, stat)

    def _start(self, slot: int, batch: list):
        """Solve a batch of (request, plan) on one slot: one plan solve, or one group solve whose
        members are enqueued concurrently, each on its own stream."""
        import torch
        st = self.streams[slot]
        items = []
        with torch.cuda.stream(st):
            for req, plan in batch:
                inp, out, bufs = self._buffers(req, plan)
                items.append((req, plan, inp, out, bufs))
        group = None
        if len(items) == 1:
            items[0][1].solve(items[0][2], items[0][3], st.cuda_stream)
        else:
            group = Group([it[1] for it in items])
            group.solve([it[2] for it in items], [it[3] for it in items], st.cuda_stream)
        ev = torch.cuda.Event()
        ev.record(st)
        now = time.perf_counter()
        for it in items:
            it[0].t_start = now
        self.batches += 1
        self.largest_batch = max(self.largest_batch, len(items))
        self.busy[slot] = ([(it[0], it[1], it[4]) for it in items], group, ev)

    def _finish(self, slot: int):
        batch, group, ev = self.busy[slot]
        t = time.perf_counter()
        for req, plan, (E, cur, den, cint, dint, stat) in batch:
            req.t_done = t
            req.result = {"current": cur.cpu().numpy() if req.n_blocks > 1 else np.zeros((len(req.energies), 0)),
                          "density": den.cpu().numpy(), "current_int": cint.cpu().numpy(),
                          "density_int": dint.cpu().numpy(), "status": stat.cpu().numpy()}
            self.plans.give(plan)
            self.done.append(req)
        if group is not None:
            group.close()
        self.busy[slot] = None

    def poll(self) -> bool:
        """Retire finished batches and admit queued requests; returns True if anything changed."""
        changed = False
        for s, item in enumerate(self.busy):
            if item is not None and item[2].query():
                self._finish(s)
                changed = True
        for s in range(len(self.busy)):
            if self.busy[s] is not None or not self.queue:
                continue
            # FIFO with skip-ahead: the first queued requests whose plans are available or fit
            batch = []
            for req in list(self.queue):
                plan = self._take_plan(self.models[req.model], req.precision)
                if plan is None:
                    continue
                self.queue.remove(req)
                batch.append((req, plan))
                if len(batch) == self.group_size:
                    break
            if batch:
                self._start(s, batch)
                changed = True
        return changed

    def close(self):
        """Free the pooled plans (call once no batch is in flight)."""
        self.plans.close()

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
        return {"completed": len(done), "submitted": len(requests),
                "rejected": len([r for r in self.rejected if r in requests]), "wall_s": t1 - t0,
                "batches": self.batches, "largest_batch": self.largest_batch,
                "energy_points_per_s": pts / (t1 - t0) if t1 > t0 else 0.0,
                "requests_per_s": len(done) / (t1 - t0) if t1 > t0 else 0.0,
                "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                "hbm_plans_bytes": int(self.plans.used), "plans_evicted": self.plans.evicted}
