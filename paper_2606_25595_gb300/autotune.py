"""Schedule autotuner for the RGF solves on the GPU; every candidate is timed, results are cached on
disk (``_autotune.json`` next to this file) keyed by shape, precision and GPU name.

Per device shape (b, N_B) and precision it picks:
* the energies in flight per plan -- the batch of every product and inverse launch, hence the tiles
  per launch and the workspace size (``best_chunk``);
* the pipeline stages of the tensor-core product kernel, where shared memory allows two sizes
  (``best_stages``).
Per group of devices it picks the pooling threshold: products of fewer than that many waves of tiles
are pooled into shared persistent launches (``best_pool_waves``).

The tensor-core tile itself is fixed by the hardware mapping: 128 rows x 48 complex columns for 6
and 7 digit planes (TMEM holds their five accumulators of 96 columns), x 64 for 4 and 2 planes
(at most four accumulators of 128).
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


def _time_plan(desc, dev_inputs, n_blocks, ec, repeats=1):
    import torch
    p = Plan(desc)
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
    st = torch.cuda.current_stream()
    p.solve(inp, o, st.cuda_stream)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(repeats):
        p.solve(inp, o, st.cuda_stream)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / repeats
    p.close()
    return ec / dt


# pipeline stages the product kernel can take per precision (the first is the default)
STAGE_CHOICES = {"emu64": (3, 2), "fp32": (3, 2), "bf16x3": (6, 4)}


def best_stages(dev_inputs: dict, b: int, n_blocks: int, precision: str, chunk: int,
                has_scattering: bool = True, refresh: bool = False) -> int:
    """Pipeline stages of the tensor-core product kernel that maximise energy-points/s for this shape
    at ``chunk`` energies in flight (0 for modes without tensor-core products)."""
    import torch
    if precision not in STAGE_CHOICES:
        return 0
    key = f"{torch.cuda.get_device_name()}|b={b}|nb={n_blocks}|{precision}|chunk={chunk}|stages"
    cache = _load()
    if key in cache and not refresh:
        return int(cache[key]["stages"])
    results = {}
    for stg in STAGE_CHOICES[precision]:
        d = make_desc(n_blocks, b, precision, chunk, has_scattering=has_scattering,
                      outputs=["current", "density"], tc_stages=stg)
        results[stg] = _time_plan(d, dev_inputs, n_blocks, chunk)
    best = max(results, key=results.get)
    cache[key] = {"stages": int(best), "energy_points_per_s": {str(k): v for k, v in results.items()}}
    _store(cache)
    return int(best)


def best_pool_waves(batch, candidates=(0, 1, 2, 4), refresh: bool = False) -> int:
    """Pooling threshold of a ``batch.UnevenBatch``'s group (waves of tiles below which products are
    pooled; 0 = never) that maximises its energy-points/s, timing one group solve per candidate.
    Leaves the best one set on the group."""
    import torch
    shapes = ",".join(f"{it['plan'].desc.block_size}x{it['plan'].desc.n_blocks}x{it['chunk']}" for it in batch.items)
    key = f"{torch.cuda.get_device_name()}|group|{batch.precision}|{shapes}|pool"
    cache = _load()
    if key in cache and not refresh:
        best = int(cache[key]["pool_waves"])
        batch.group.set_pool_waves(best)
        return best
    results = {}
    for w in candidates:
        batch.group.set_pool_waves(w)
        batch.launch()  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.launch()
        torch.cuda.synchronize()
        results[w] = batch.n_energies / (time.perf_counter() - t0)
    best = max(results, key=results.get)
    batch.group.set_pool_waves(best)
    cache[key] = {"pool_waves": int(best), "energy_points_per_s": {str(k): v for k, v in results.items()}}
    _store(cache)
    return int(best)
