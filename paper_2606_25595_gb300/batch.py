"""Uneven batches: several devices of different block size b and slice count N_B, each with its own
energy grid, solved together and replayed as one CUDA graph.

Energies are independent (Sec. II-A: Eq. 2 is solved per energy), so devices of different shapes
share the GPU without any exchange.  Each device gets its own plan (workspace sized for its shape and
energies in flight).  With ``grouped`` (the default) the plans form a ``qtx_rgf_group``: one call
solves every device, each on its own stream, and at every step the tensor-core products of all
devices run as one persistent kernel launch over the union of their tiles.  Otherwise each device's
solve is launched on its own stream.  ``capture()`` records one launch of the whole batch into a CUDA
graph and ``replay()`` replays it.  Solves with a per-energy status output make no host
synchronisation, so they capture cleanly.  This module only marshals arguments and orders launches;
every step of the solves runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import Group, Outputs, Plan, make_desc, upload


class UnevenBatch:
    """Resident inputs, plans and outputs of a list of ``workloads``-style device dicts.

    ``chunks``: energies in flight per device (default: all of the device's energies).
    ``stages``, ``ctas``: per-device schedule of the tensor-core product kernel (``make_desc``'s
    ``tc_stages``, ``tc_ctas``; default 0 = the kernel's own).
    ``outputs``: names as in ``make_desc``; per-energy arrays and integrals are kept on the device."""

    def __init__(self, devs: list, precision: str = "fp32", chunks=None, refine_max_iter: int = 2,
                 refine_tol: float = 0.0, outputs=("current", "density", "integrals"), grouped: bool = True,
                 stages=None, ctas=None):
        import torch
        self.devs = devs
        self.grouped = grouped
        self.precision = precision
        self.items = []
        for k, dev in enumerate(devs):
            nb, b = dev["n_blocks"], dev["block_size"]
            E = np.asarray(dev["energies"], dtype=np.float64)
            ne = E.size
            ec = ne if chunks is None else int(min(chunks[k], ne))
            want = [o for o in outputs if not (o in ("contact", "transmission") and not dev.get("leads"))]
            din = upload(dev, E)
            desc = make_desc(nb, b, precision, ec, refine_max_iter, has_S=dev.get("S_diag") is not None,
                             has_scattering=dev.get("SigR") is not None, leads=bool(dev.get("leads")),
                             outputs=want, refine_tol=refine_tol,
                             tc_stages=0 if stages is None else int(stages[k]),
                             tc_ctas=0 if ctas is None else int(ctas[k]))
            plan = Plan(desc)
            o = Outputs()
            bufs = {}
            shapes = {"current": (ne, max(nb - 1, 1)), "density": (ne, nb), "contact": (ne, 2),
                      "transmission": (ne,)}
            for name in want:
                if name == "integrals":
                    bufs["current_int"] = torch.zeros(max(nb - 1, 1), dtype=torch.float64, device="cuda")
                    bufs["density_int"] = torch.zeros(nb, dtype=torch.float64, device="cuda")
                    o.current_int = bufs["current_int"].data_ptr() if nb > 1 else None
                    o.density_int = bufs["density_int"].data_ptr()
                elif name in shapes:
                    bufs[name] = torch.empty(shapes[name], dtype=torch.float64, device="cuda")
                    setattr(o, name, bufs[name].data_ptr())
                else:
                    shp = (ne, nb if "diag" in name else nb - 1, b, b)
                    bufs[name] = torch.empty(shp, dtype=torch.complex128, device="cuda")
                    setattr(o, name, bufs[name].data_ptr())
            bufs["status"] = torch.zeros(ne, dtype=torch.int32, device="cuda")
            o.status_per_energy = bufs["status"].data_ptr()
            self.items.append(dict(plan=plan, din=din, out=o, bufs=bufs, chunk=ec, n_energies=ne))
        self.streams = [torch.cuda.Stream() for _ in devs]
        self.group = Group([it["plan"] for it in self.items]) if grouped else None
        self.graph = None

    @property
    def n_energies(self) -> int:
        return sum(it["n_energies"] for it in self.items)

    def launch(self):
        """Enqueue every device's solve, forked from and joined back to the current stream: one group
        solve (pooled product launches), or one solve per device on its own stream."""
        import torch
        cur = torch.cuda.current_stream()
        if self.group is not None:
            self.group.solve([it["din"]["_inputs"] for it in self.items], [it["out"] for it in self.items],
                             cur.cuda_stream)
            return
        for it, s in zip(self.items, self.streams):
            s.wait_stream(cur)
            it["plan"].solve(it["din"]["_inputs"], it["out"], s.cuda_stream)
        for s in self.streams:
            cur.wait_stream(s)

    def capture(self):
        """Record one ``launch()`` into a CUDA graph (after one eager warm-up launch)."""
        import torch
        self.launch()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        # a group solve enqueues from one host thread per device into the capturing streams
        with torch.cuda.graph(g, stream=torch.cuda.Stream(), capture_error_mode="thread_local"):
            self.launch()
        torch.cuda.synchronize()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def results(self) -> list:
        """Per device: a dict of numpy arrays (outputs and per-energy status)."""
        import torch
        torch.cuda.synchronize()
        return [{k: v.cpu().numpy() for k, v in it["bufs"].items()} for it in self.items]

    def close(self):
        self.graph = None
        if self.group is not None:
            self.group.close()
            self.group = None
        for it in self.items:
            it["plan"].close()
