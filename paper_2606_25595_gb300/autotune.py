"""Schedule autotuner: picks the number of energies in flight per plan (the batch of every product
and inverse launch, hence the number of CTAs per launch and the workspace size) for a device shape
(b, N_B) and precision, by timing one solve per candidate on the GPU.  Results are cached on disk
(``_autotune.json`` next to this file) keyed by shape, precision and GPU name.

The kernels' tiles are fixed by the hardware mapping (128 x 48 complex output tiles for the tensor-core
engine, 128/64/32-square tiles for the SIMT GEMM chosen from M, N); the schedule parameter that varies
with (b, N_B) is how many energies each launch covers.
"""
from __future__ import annotations

import json
import os
import time

from . import Inputs, Outputs, Plan, footprint, make_desc

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "_autotune.json")


def _load():
    if os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def _store(c):
    try:
        with open(CACHE, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
    except OSError:
        pass


def best_chunk(dev_inputs: dict, b: int, n_blocks: int, precision: str, n_energies: int,
               candidates=(16, 32, 64, 128, 256), budget_bytes: int | None = None,
               has_scattering: bool = True, refresh: bool = False) -> int:
    """Energies in flight that maximise energy-points/s for this shape, measured on ``dev_inputs``
    (an ``upload``-style dict whose energies array holds at least max(candidates) energies)."""
    import torch
    key = f"{torch.cuda.get_device_name()}|b={b}|nb={n_blocks}|{precision}|scat={int(has_scattering)}"
    cache = _load()
    if key in cache and not refresh:
        return int(cache[key]["chunk"])
    free, _ = torch.cuda.mem_get_info()
    budget = budget_bytes if budget_bytes is not None else int(free * 0.5)
    results = {}
    st = torch.cuda.current_stream()
    for ec in candidates:
        ec = min(ec, n_energies)
        if ec in results:
            continue
        d = make_desc(n_blocks, b, precision, ec, has_scattering=has_scattering,
                      outputs=["current", "density"])
        if footprint(d) > budget:
            continue
        p = Plan(d)
        inp = Inputs.from_buffer_copy(dev_inputs["_inputs"])
        inp.n_energies = ec
        inp.n_blocks = n_blocks
        cur = torch.empty((ec, max(n_blocks - 1, 1)), dtype=torch.float64, device="cuda")
        den = torch.empty((ec, n_blocks), dtype=torch.float64, device="cuda")
        stat = torch.zeros(ec, dtype=torch.int32, device="cuda")
        o = Outputs()
        o.current = cur.data_ptr() if n_blocks > 1 else None
        o.density = den.data_ptr()
        o.status_per_energy = stat.data_ptr()
        p.solve(inp, o, st.cuda_stream)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.solve(inp, o, st.cuda_stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        results[ec] = ec / dt
        p.close()
    best = max(results, key=results.get) if results else min(candidates)
    cache[key] = {"chunk": int(best), "energy_points_per_s": {str(k): v for k, v in results.items()}}
    _store(cache)
    return int(best)
