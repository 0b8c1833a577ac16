#!/usr/bin/env python
"""Throughput benchmark of the RGF selected inversion on GB300: prints ONE JSON line.

Workload (default): the batched mixed-precision device -- b = 256 complex blocks, N_B = 64 slices,
N_E = 512 energies on [-2, 2], dense random Hermitian diagonal blocks, coupling blocks of variance
0.3/b, block-diagonal scattering self-energies (seeded synthetic data, see ``workloads``).  One
step = one ``qtx_rgf_solve`` of all 512 energies (forward and backward sweeps, G^R/G^< diagonal
blocks kept resident in HBM, per-slice current and density and their energy integrals), in the
emulated-FP64 mode (tensor-core digit products) unless ``--precision`` says otherwise.

Also measured in the same run: the plain FP64 path on a subset of the same energies, the
product kernel's live duration (CUDA events on the solve stream) for the roofline, the end-to-end
rate through the C ABI with host buffers, the CPU FP64 oracle on a bounded sample (and the error of
the GPU result at those energies), and the SM clocks during the timed region.

``--impl reference`` times the CPU FP64 oracle instead (bounded sample per step).
Multi-GPU (torchrun): every rank solves its own 512-energy batch on its own GPU with no
collective in the data path (weak scaling); timing is max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RGF energy-points/s vs FP64 path at <=1e-6 rel. current error; p50/p99 latency"
UNIT = "energy-points/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="emu64", choices=["emu64", "fp32", "bf16x3", "fp64"])
    ap.add_argument("--chunk", type=int, default=512, help="energies in flight per chunk (512: all 512 energies of the mixed workload in one chunk, 6144 product tiles = 40.4 waves on 152 SMs)")
    ap.add_argument("--block", type=int, default=256)
    ap.add_argument("--slices", type=int, default=64)
    ap.add_argument("--energies", type=int, default=512)
    ap.add_argument("--fp64-energies", type=int, default=16, help="energies for the FP64 comparison (0 = skip)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU oracle sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="mixed", choices=["mixed", "mixed_bt", "strip", "uneven", "ozaki", "serving", "nrl", "wsolve"],
                    help="mixed: b=256 N_B=64 N_E=512 (default); mixed_bt: the same with block-tridiagonal "
                         "scattering self-energies; strip: W=16 strip FP64 with contacts; "
                         "uneven: 8 devices x 128 energies in one CUDA graph; ozaki: b=1024 N_B=32 "
                         "emulated FP64 (subset of the 256 energies); serving: Poisson request stream; "
                         "nrl: b=3408 N_B=10 (the paper's NR-L shape), per-energy self-energies streamed from host; "
                         "wsolve: screened-Coulomb system b=256 N_B=32, 64 energies (assembly + one selected solve for B^< and B^>)")
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--group", type=int, default=4, help="serving: requests admitted together as one group solve")
    ap.add_argument("--serving-solo", action="store_true", help="serving: also run the stream without batching")
    ap.add_argument("--refine-tol", type=float, default=2.0 ** -12,
                    help="mixed workloads: an energy stops its Newton sweeps once ||I - A X||_F <= this "
                         "(the next residual is then <= its square, 2^-24, below the digit products' error); "
                         "0 = always 2 sweeps")
    ap.add_argument("--modes", default="fp32,bf16x3",
                    help="mixed workloads: other precision modes timed on the same workload after the headline "
                         "(one solve each, all energies), with their error against the oracle sample")
    ap.add_argument("--no-modes", action="store_true")
    ap.add_argument("--no-others", action="store_true",
                    help="mixed workload: skip the secondary measurements (strip, uneven batch, b = 1024 device, serving)")
    ap.add_argument("--storage-bits", type=int, default=0,
                    help="mixed workloads: keep the left-connected blocks in FPX of this many bits (0 = off)")
    ap.add_argument("--tc-stages", type=int, default=0,
                    help="mixed workloads: pipeline stages of the tensor-core product kernel (0 = its default)")
    ap.add_argument("--tc-ctas", type=int, default=0,
                    help="mixed workloads: persistent CTAs per product launch (0 = one per SM)")
    return ap.parse_args()


def dist_init():
    from paper_2606_25595_gb300 import dist as D
    return D.init()


def barrier(ws):
    from paper_2606_25595_gb300 import dist as D
    D.barrier(ws)


def max_over_ranks(x, ws):
    from paper_2606_25595_gb300 import dist as D
    return D.max_over_ranks(x, ws)


def source_hash(path):
    """First 16 hex digits of the SHA-256 of a CUDA source with its comments and blank lines removed
    (a comment edit leaves the kernel, and so the counters taken on it, unchanged)."""
    import hashlib
    import re
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", l).rstrip() for l in text.splitlines()]
    code = "\n".join(l for l in lines if l.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def captured_traffic(energies_per_launch):
    """DRAM bytes per product-kernel launch from the committed ncu capture, scaled by the energies a
    launch processes (traffic grows in proportion: each energy's planes are read once).  None when
    the kernel source changed since the capture."""
    cap = os.path.join(ROOT, "profiles", "k_tc_gemm_emu64_b256_e64.txt")
    src = os.path.join(ROOT, "paper_2606_25595_gb300", "csrc", "tc_engine.cu")
    if not (os.path.exists(cap) and os.path.exists(src)):
        return None, None
    txt = open(cap).read()
    h = source_hash(src)
    per = None
    same = False
    for line in txt.splitlines():
        if line.startswith("source_code_sha256_16:"):
            same = line.split()[1] == h
        if line.startswith("dram_bytes_per_energy:"):
            per = float(line.split()[1])
    if not same or per is None:
        return None, per
    return per * energies_per_launch, per


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", self.uuid, f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_oracle_sample(dev, budget_s, idx_pool):
    """Time the FP64 oracle on host cores for as many energies of the pool as fit the budget."""
    import oracle as O
    t0 = time.perf_counter()
    done, res = [], {}
    for k in idx_pool:
        r = O.rgf_energy(float(dev["energies"][k]), dev, int(k))
        res[int(k)] = (r["current"], r["density"])
        done.append(int(k))
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return done, res, dt


def run_reference(args):
    import workloads as W
    dev = W.random_device(args.block, args.slices, n_energies=args.energies, seed=0,
                          offdiag_sigma=args.workload == "mixed_bt")
    per_step = 2
    import numpy as np
    pool = list(np.linspace(0, args.energies - 1, per_step * (args.steps + args.warmup)).astype(int))
    for w in range(args.warmup):
        cpu_oracle_sample(dev, 1e9, pool[w * per_step:(w + 1) * per_step])
    t = 0.0
    n = 0
    for s in range(args.steps):
        sl = pool[(args.warmup + s) * per_step:(args.warmup + s + 1) * per_step]
        done, _, dt = cpu_oracle_sample(dev, 1e9, sl)
        t += dt
        n += len(done)
    value = n / t
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"random BT device b={args.block} N_B={args.slices} N_E={args.energies} on [-2,2], "
                                   "block-diagonal scattering self-energies (seed 0)",
                       "global_batch": args.energies, "precision": "fp64-oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} energies of the {args.energies}-energy grid per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _line(args, metric_value, ms_per_step, workload, precision, extra):
    line = {"metric": METRIC, "value": metric_value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"emu64": "bf16-digits(tcgen05)+df32", "fp32": "c64",
                                           "fp64": "c128", "bf16x3": "bf16-digits(tcgen05)+df32"}[precision],
            "data": "synthetic", "config": {"workload": workload, "precision": precision}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def _solve_setup(q, dev, precision, chunk, outs, energies=None):
    import torch
    E = dev["energies"] if energies is None else energies
    din = q.upload(dev, E)
    nb, b, ne = dev["n_blocks"], dev["block_size"], len(E)
    want = [o for o in outs if not (o in ("contact", "transmission") and not dev.get("leads"))]
    desc = q.make_desc(nb, b, precision, min(chunk, ne), 2, has_S=dev.get("S_diag") is not None,
                       has_scattering=dev.get("SigR") is not None, leads=bool(dev.get("leads")), outputs=want)
    plan = q.Plan(desc)
    o = q.Outputs()
    bufs = {}
    shapes = {"current": (ne, max(nb - 1, 1)), "density": (ne, nb), "contact": (ne, 2), "transmission": (ne,)}
    for k in want:
        if k == "integrals":
            bufs["current_int"] = torch.zeros(max(nb - 1, 1), dtype=torch.float64, device="cuda")
            bufs["density_int"] = torch.zeros(nb, dtype=torch.float64, device="cuda")
            o.current_int, o.density_int = bufs["current_int"].data_ptr(), bufs["density_int"].data_ptr()
        elif k in shapes:
            bufs[k] = torch.empty(shapes[k], dtype=torch.float64, device="cuda")
            setattr(o, k, bufs[k].data_ptr())
        else:
            shp = (ne, nb if "diag" in k else nb - 1, b, b)
            bufs[k] = torch.empty(shp, dtype=torch.complex128, device="cuda")
            setattr(o, k, bufs[k].data_ptr())
    bufs["status"] = torch.zeros(ne, dtype=torch.int32, device="cuda")
    o.status_per_energy = bufs["status"].data_ptr()
    return plan, din, o, bufs


def _timed(step, steps, warmup):
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


# energies in flight per device of the uneven workload, as the autotuner picks them on this GPU
UNEVEN_CHUNKS = [128, 128, 128, 128, 64, 128, 128, 128]


def secondary_workloads(q, W, steps=3, warmup=2):
    """The W=16 strip (FP64, contacts, one solve replayed from a CUDA graph), the uneven 8-device batch
    (FP32 products on the tensor cores, one group solve replayed from a CUDA graph), the b = 1024
    device (emulated FP64, 16 energies), each timed with CUDA events after warm-up, with the strip's
    error against the CPU oracle (all 64 energies); and a short serving run (config 5, wall clock)."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2606_25595_gb300.batch import UnevenBatch
    out = {}
    st = torch.cuda.current_stream()
    dev = W.strip(**W.STRIP_CFG)
    keys = ("current", "density", "contact", "transmission")
    sb = UnevenBatch([dev], "fp64", [64], outputs=keys + ("integrals",), grouped=False)
    sb.launch()
    eager = sb.results()[0]
    sb.capture()
    ms = _timed(sb.replay, 20, 3)
    got = sb.results()[0]
    ref = O.solve(dev, keep_blocks=False)
    out["strip_config1_fp64"] = {
        "value": 64 * 20 / (ms / 1e3), "unit": UNIT,
        "workload": "W=16 strip b=16 N_B=32 N_E=64 [-3.5,3.5] eta=1e-6, Sancho-Rubio contacts; "
                    "one solve of all 64 energies replayed from a CUDA graph",
        "replay_equals_eager": all(bool(np.array_equal(eager[k], got[k])) for k in keys),
        "error_vs_oracle": {k: float(np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max()) for k in keys}}
    sb.close()
    devs = W.uneven_batch(n_energies=128)
    ub = UnevenBatch(devs, "fp32", UNEVEN_CHUNKS)
    ub.capture()
    ms = _timed(ub.replay, steps, warmup)
    out["uneven_config3_fp32"] = {
        "value": ub.n_energies * steps / (ms / 1e3), "unit": UNIT,
        "workload": "8 random BT devices (N_B, b) = " + ", ".join(f"({d['n_blocks']},{d['block_size']})" for d in devs)
                    + ", 128 energies each, one group solve replayed from a CUDA graph",
        "status_ok": all(bool(np.all(r["status"] == 0)) for r in ub.results())}
    ub.close()
    torch.cuda.empty_cache()
    # config 4: b = 1024, N_B = 32, emulated FP64 (seven digits), 16 of its 256 energies
    d4 = W.random_device(W.OZAKI_CFG["b"], W.OZAKI_CFG["n_blocks"], n_energies=W.OZAKI_CFG["n_energies"], seed=0)
    sub = np.linspace(0, W.OZAKI_CFG["n_energies"] - 1, 16).astype(int)
    plan, din, o, bufs = _solve_setup(q, d4, "emu64", 16, ["current", "density"], energies=d4["energies"][sub])
    ms = _timed(lambda: plan.solve(din["_inputs"], o, st.cuda_stream), 1, 1)
    out["ozaki_config4_emu64"] = {
        "value": 16 / (ms / 1e3), "unit": UNIT,
        "workload": "random BT device b=1024 N_B=32, 16 of its 256 energies on [-2,2], emulated FP64 (7 digit planes)",
        "status_ok": bool(torch.all(bufs["status"] == 0).item())}
    plan.close()
    torch.cuda.empty_cache()
    # config 5: 40 requests at 200/s (saturating), then 20 at 0.7 x the measured capacity
    sat, sub, lam, _ = serving_runs(q, W, 40, 4)
    keep = ("completed", "submitted", "rejected", "requests_per_s", "energy_points_per_s", "p50_s", "p99_s", "wall_s",
            "plans_evicted")
    out["serving_config5"] = {
        "value": sat["energy_points_per_s"], "unit": UNIT,
        "workload": "40 Poisson requests at 200/s (b in {64,128,256,512}, N_B~U[16,96], N_E in {32,64,128}, "
                    "complex64 / emulated-FP64), admitted in groups of 4 on 4 streams",
        "saturated": {k: sat[k] for k in keep if k in sat},
        f"at_0.7_capacity_{lam:.2f}_per_s": {k: sub[k] for k in keep if k in sub}}
    torch.cuda.empty_cache()
    return out


def run_strip(args, q, W):
    """W=16 strip, b=16, N_B=32, 64 energies, Sancho-Rubio contacts, plain FP64."""
    import numpy as np
    import torch
    import oracle as O
    dev = W.strip(**W.STRIP_CFG)
    prec = args.precision if args.precision != "emu64" else "fp64"
    plan, din, o, bufs = _solve_setup(q, dev, prec, 64, ["GR_diag", "GL_diag", "current", "density",
                                                         "contact", "transmission", "integrals"])
    st = torch.cuda.current_stream()
    launches0 = q.kernel_launches()
    ms = _timed(lambda: plan.solve(din["_inputs"], o, st.cuda_stream), args.steps, args.warmup)
    launches = (q.kernel_launches() - launches0) * args.steps // (args.steps + args.warmup)
    value = 64 * args.steps / (ms / 1e3)
    t0 = time.perf_counter()
    ref = O.solve(dev, keep_blocks=False)
    tc = time.perf_counter() - t0
    err = {k: float(np.abs(bufs[k].cpu().numpy() - ref[k]).max() / np.abs(ref[k]).max())
           for k in ("current", "density", "contact", "transmission")}
    _line(args, value, ms / args.steps, "W=16 strip b=16 N_B=32 N_E=64 [-3.5,3.5] eta=1e-6, Sancho-Rubio "
          "contacts, onsite U[-0.25,0.25]", prec,
          {"gpu_launches": int(launches), "status_ok": bool(torch.all(bufs["status"] == 0).item()),
           "cpu_baseline": {"value": 64 / tc, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": "all 64 energies"},
           "error_vs_oracle": err})


def _gemm_roofline(prof, peak):
    """Roofline of the product kernel from a plan's GEMM profile: algorithmic flops (8 M N K per
    complex product) over the kernel's live time against ``peak``, and the tensor pipe's flops (every
    digit product) beside them."""
    if not prof["ms"]:
        return {"bound": "tensor", "achieved": None, "peak": peak, "unit": "TFLOP/s", "frac": None}
    sec = prof["ms"] / 1e3
    ach, pipe = prof["useful_flops"] / sec / 1e12, prof["pipe_flops"] / sec / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak if peak else None,
            "achieved_counts": "algorithmic flops: 8 M N K per complex product (complex FP64-equivalent)",
            "pipe_achieved": pipe, "pipe_frac": pipe / peak if peak else None}


def run_ozaki(args, q, W):
    """b=1024, N_B=32 (blocks as in the mixed workload), emulated FP64, a subset of the 256 energies."""
    import numpy as np
    import torch
    cfg = W.OZAKI_CFG
    ne = args.energies if args.energies != 512 else 32
    dev = W.random_device(cfg["b"], cfg["n_blocks"], n_energies=cfg["n_energies"], seed=0)
    idx = np.linspace(0, cfg["n_energies"] - 1, ne).astype(int)
    plan, din, o, bufs = _solve_setup(q, dev, args.precision, min(args.chunk, 16), ["current", "density", "integrals"],
                                      energies=dev["energies"][idx])
    st = torch.cuda.current_stream()
    plan.set_profiling(True)
    ms = _timed(lambda: plan.solve(din["_inputs"], o, st.cuda_stream), args.steps, args.warmup)
    prof = plan.gemm_profile()
    value = ne * args.steps / (ms / 1e3)
    peaks, _ = measured_peaks()
    _line(args, value, ms / args.steps, f"random BT device b=1024 N_B=32, {ne} of 256 energies on [-2,2]",
          args.precision, {"status_ok": bool(torch.all(bufs["status"] == 0).item()),
                           "roofline": _gemm_roofline(prof, peaks.get("bf16_tflops_sustained"))})


def run_nrl(args, q, W):
    """b=3408, N_B=10 (the paper's NR-L block shape), emulated FP64, energy-dependent self-energies
    held in pinned host memory and streamed slice by slice (sigma_stream); one chunk of all energies
    per step, H2D copies of the self-energies inside the timed region."""
    import torch
    cfg = W.NRL_CFG
    ne = cfg["n_energies"]
    dev = W.nrl_device(cfg["b"], cfg["n_blocks"], ne, cfg["e_lo"], cfg["e_hi"])
    nb, b = cfg["n_blocks"], cfg["b"]
    din = q.upload(dev, sigma_host=True)
    outs = ["current", "density", "integrals"]
    desc = q.make_desc(nb, b, args.precision, ne, 2, has_scattering=True, energy_dependent_sigma=True,
                       outputs=outs, sigma_stream=True, storage_bits=args.storage_bits)
    plan = q.Plan(desc)
    o = q.Outputs()
    cur = torch.empty((ne, nb - 1), dtype=torch.float64, device="cuda")
    den = torch.empty((ne, nb), dtype=torch.float64, device="cuda")
    cint = torch.zeros(nb - 1, dtype=torch.float64, device="cuda")
    dint = torch.zeros(nb, dtype=torch.float64, device="cuda")
    stat = torch.zeros(ne, dtype=torch.int32, device="cuda")
    o.current, o.density = cur.data_ptr(), den.data_ptr()
    o.current_int, o.density_int = cint.data_ptr(), dint.data_ptr()
    o.status_per_energy = stat.data_ptr()
    st = torch.cuda.current_stream()
    plan.set_profiling(True)
    ms = _timed(lambda: plan.solve(din["_inputs"], o, st.cuda_stream), args.steps, args.warmup)
    prof = plan.gemm_profile()
    value = ne * args.steps / (ms / 1e3)
    peaks, _ = measured_peaks()
    useful = 136.0 * b ** 3 * nb * ne * args.steps / (ms / 1e3) / 1e12
    _line(args, value, ms / args.steps, f"NR-L-shaped device b={b} N_B={nb}, {ne} energies per step, "
          "per-energy scattering self-energies streamed from pinned host memory", args.precision,
          {"status_ok": bool(torch.all(stat == 0).item()),
           "plan_bytes": q.footprint(desc), "host_sigma_bytes_per_step": 2 * ne * nb * b * b * 16,
           "useful_fp64_equiv_tflops": useful,
           "roofline": _gemm_roofline(prof, peaks.get("bf16_tflops_sustained"))})


def run_wsolve(args, q, W):
    """Screened-Coulomb system (Table I, W row): per step, assemble M = I - V P^R and B^<> = V P^<>
    V^H for all energies and solve M X M^H = B^< and B^> (one selected solve with two right-hand
    sides sharing the retarded sweep).  Error against the oracle on a small system of the same
    generator (b=64, N_B=6, 2 energies)."""
    import time
    import numpy as np
    import torch
    from oracle import wsys
    cfg = W.WSYS_CFG
    b, nb, ne = cfg["b"], cfg["n_blocks"], cfg["n_energies"]
    w = W.w_system(b, nb, n_energies=ne, seed=0)
    st = torch.cuda.current_stream()
    ws = q.WSystem(w, args.precision, max_energies_in_flight=min(args.chunk, ne))
    step = lambda: ws.run(st.cuda_stream)
    for _ in range(args.warmup):
        step()
    launches0 = q.kernel_launches()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(st)
    ws.plan.set_profiling(True)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = q.kernel_launches() - launches0
    prof = ws.plan.gemm_profile()
    status_ok = bool(torch.all(ws.res["status"] == 0).item())
    ms = e0.elapsed_time(e1)
    small = W.w_system(64, 6, n_energies=2, seed=1)
    got = q.solve_w(small, args.precision)
    err = 0.0
    for k in range(2):
        PR = (small["PR_diag"][k], small["PR_upper"][k], small["PR_lower"][k])
        M = wsys.assemble(small["V_diag"], small["V_upper"], PR, (small["PL_diag"][k], small["PL_upper"][k]),
                          (small["PG_diag"][k], small["PG_upper"][k]))
        ref = wsys.solve(M, (M["BL_diag"], M["BL_upper"]), (M["BG_diag"], M["BG_upper"]))
        for key in ("XL_diag", "XG_diag", "XR_diag"):
            err = max(err, float(np.linalg.norm(got[key][k] - ref[key]) / np.linalg.norm(ref[key])))
    value = ne * args.steps / (ms / 1e3)
    peaks, _ = measured_peaks()
    _line(args, value, ms / args.steps, f"screened-Coulomb system b={b} N_B={nb}, {ne} energies per step "
          "(assembly of M = I - V P^R, B^<> = V P^<> V^H and the selected solve for B^< and B^>; inputs resident)",
          args.precision,
          {"status_ok": status_ok, "wall_s_per_step": wall / args.steps, "gpu_launches": int(launches),
           "product_kernel_share": prof["ms"] / ms if ms else None,
           "roofline": _gemm_roofline(prof, peaks.get("bf16_tflops_sustained")),
           "error_vs_oracle": {"system": "b=64 N_B=6, 2 energies, same generator", "max_rel_frobenius": err}})


def run_uneven(args, q, W):
    """8 devices (N_B in 16..128, b in 128..512), 128 energies each, all solves captured in one CUDA
    graph (one stream per device), energies in flight per device from the autotuner."""
    import numpy as np
    import torch
    from paper_2606_25595_gb300 import autotune
    from paper_2606_25595_gb300.batch import UnevenBatch
    prec = args.precision if args.precision != "emu64" else "fp32"
    devs = W.uneven_batch(n_energies=128)
    chunks, stages = [], []
    for dev in devs:
        din = q.upload(dev)
        chunks.append(autotune.best_chunk(din, dev["block_size"], dev["n_blocks"], prec, 128,
                                          budget_bytes=24 << 30))
        stages.append(autotune.best_stages(din, dev["block_size"], dev["n_blocks"], prec, chunks[-1]))
        del din
    ub = UnevenBatch(devs, prec, chunks, stages=stages)
    pool = autotune.best_pool_waves(ub)
    captured = True
    try:
        ub.capture()
    except Exception as ex:  # capture refused: fall back to direct launches, say so
        captured = False
        sys.stderr.write(f"graph capture failed: {ex}\n")
    torch.cuda.synchronize()
    step = ub.replay if captured else ub.launch
    ms = _timed(step, args.steps, args.warmup)
    ne_total = ub.n_energies
    ok = all(bool(np.all(r["status"] == 0)) for r in ub.results())
    _line(args, ne_total * args.steps / (ms / 1e3), ms / args.steps,
          "8 random BT devices (N_B, b) = " + ", ".join(f"({d['n_blocks']},{d['block_size']})" for d in devs)
          + ", 128 energies each", prec,
          {"status_ok": ok, "cuda_graph": captured, "energies_in_flight": chunks, "tc_stages": stages,
           "pool_waves": pool})


def serving_runs(q, W, n_requests, group, solo=False):
    """Poisson request stream (mean 200/s): b in {64,128,256,512}, N_B ~ U[16,96], N_E in {32,64,128},
    complex64 / emulated-FP64 tags; then the same at 0.7 x the measured capacity.  Returns the
    saturated run, the run at 0.7 x capacity with its rate, and (solo) the saturated run without
    batching."""
    import numpy as np
    from paper_2606_25595_gb300 import serve
    models = {}
    for b in (64, 128, 256, 512):
        models[f"b{b}"] = serve.DeviceModel(W.random_device(b, 96, n_energies=1, seed=500 + b), f"b{b}")

    def reqs(n, rate, seed):
        out = []
        for r in W.serving_requests(n, rate_hz=rate, seed=seed):
            E = np.linspace(-2.0, 2.0, r["n_energies"])
            out.append(serve.Request(len(out), f"b{r['b']}", r["n_blocks"], E,
                                     "emu64" if r["precision"] == "emu64" else "fp32", 0.0, 0.0,
                                     r["t_arrival"] - 0.0))
        t0 = out[0].t_arrival if out else 0.0
        for r in out:
            r.t_arrival -= t0
        return out

    def server(group):
        srv = serve.Server(models, slots=4, group_size=group)
        srv.warm(("emu64", "fp32"), per_key=group)
        # warm every kernel once
        srv.run([serve.Request(0, "b64", 16, np.linspace(-1, 1, 4), "emu64"),
                 serve.Request(1, "b64", 16, np.linspace(-1, 1, 4), "fp32")])
        return srv

    def run(group, requests):
        srv = server(group)
        stats = srv.run(requests, time_limit=300.0)
        srv.close()
        return stats

    sat = run(group, reqs(n_requests, 200.0, 1))
    alone = run(1, reqs(n_requests, 200.0, 1)) if (group > 1 and solo) else None
    lam = max(0.7 * sat["requests_per_s"], 0.05)
    sub = run(group, reqs(max(n_requests // 2, 10), lam, 2))
    return sat, sub, lam, alone


def run_serving(args, q, W):
    """Config 5 alone (see serving_runs)."""
    sat, sub, lam, solo = serving_runs(q, W, args.requests, args.group, args.serving_solo)
    _line(args, sat["energy_points_per_s"], 1e3 * sat["wall_s"],
          "served RGF requests: Poisson arrivals, b in {64,128,256,512}, N_B~U[16,96], N_E in "
          "{32,64,128}, complex64/emulated-FP64 tags", "emu64",
          {"serving": {"saturated_200_per_s": sat, f"at_0.7_capacity_{lam:.2f}_per_s": sub,
                       "saturated_without_batching": solo, "slots": 4, "group_size": args.group}})


def main():
    args = parse()
    rank, ws, lr = dist_init()
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if args.workload not in ("mixed", "mixed_bt"):
        from paper_2606_25595_gb300 import build as qbuild
        qbuild.build()
        import paper_2606_25595_gb300 as q
        import workloads as W
        {"strip": run_strip, "uneven": run_uneven, "ozaki": run_ozaki, "serving": run_serving,
         "nrl": run_nrl, "wsolve": run_wsolve}[args.workload](args, q, W)
        return
    import numpy as np
    import torch

    from paper_2606_25595_gb300 import build as qbuild
    qbuild.build()
    import paper_2606_25595_gb300 as q
    import workloads as W

    torch.cuda.set_device(lr)
    bt = args.workload == "mixed_bt"
    dev = W.random_device(args.block, args.slices, n_energies=args.energies, seed=0, offdiag_sigma=bt)
    nb, b, ne = args.slices, args.block, args.energies
    din = q.upload(dev)
    outs = ["GR_diag", "GL_diag", "current", "density", "integrals"]
    desc = q.make_desc(nb, b, args.precision, min(args.chunk, ne), refine_max_iter=2,
                       has_scattering=True, outputs=outs, offdiag_sigma=bt, storage_bits=args.storage_bits,
                       refine_tol=args.refine_tol, tc_stages=args.tc_stages, tc_ctas=args.tc_ctas)
    plan = q.Plan(desc)
    cd = torch.device("cuda")
    GR = torch.empty((ne, nb, b, b), dtype=torch.complex128, device=cd)
    GL = torch.empty((ne, nb, b, b), dtype=torch.complex128, device=cd)
    cur = torch.empty((ne, nb - 1), dtype=torch.float64, device=cd)
    den = torch.empty((ne, nb), dtype=torch.float64, device=cd)
    cint = torch.empty(nb - 1, dtype=torch.float64, device=cd)
    dint = torch.empty(nb, dtype=torch.float64, device=cd)
    stat = torch.zeros(ne, dtype=torch.int32, device=cd)
    o = q.Outputs()
    o.GR_diag, o.GL_diag = GR.data_ptr(), GL.data_ptr()
    o.current, o.density = cur.data_ptr(), den.data_ptr()
    o.current_int, o.density_int = cint.data_ptr(), dint.data_ptr()
    o.status_per_energy = stat.data_ptr()
    stream = torch.cuda.current_stream()

    def step():
        plan.solve(din["_inputs"], o, stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # ---------------------------------------------------------------- timed region (device)
    sampler = ClockSampler(str(torch.cuda.get_device_properties(lr).uuid)
                           if str(torch.cuda.get_device_properties(lr).uuid).startswith("GPU-")
                           else "GPU-" + str(torch.cuda.get_device_properties(lr).uuid))
    plan.set_profiling(True)
    barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    l0 = q.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    launches = q.kernel_launches() - l0
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    prof = plan.gemm_profile()
    plan.set_profiling(False)
    ms_max = max_over_ranks(ms, ws)
    status_ok = bool(torch.all(stat == 0).item())
    value = ws * ne * args.steps / (ms_max / 1e3)

    # ---------------------------------------------------------------- roofline of the product kernel
    peaks, peak_src = measured_peaks()
    if args.precision in ("emu64", "bf16x3"):
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        bound, kernel = "tensor", "k_tc_gemm (tcgen05 bf16 digit products)"
    elif args.precision == "fp32":
        peak, bound, kernel = 69.7, "alu", "k_gemm<float> (SIMT FFMA)"
    else:
        peak, bound, kernel = 1.1, "alu", "k_gemm<double> (SIMT DFMA)"
    # achieved: the method's own flops (8 M N K per complex product, 136 b^3 per slice) over the
    # kernel's live launch time; the tensor pipe's flops (every digit product) are reported beside
    avg_ms = prof["ms"] / max(prof["launches"], 1)
    sec = avg_ms / 1e3
    n_l = max(prof["launches"], 1)
    achieved = (prof["useful_flops"] / n_l) / sec / 1e12 if prof["launches"] else None
    pipe = (prof["pipe_flops"] / n_l) / sec / 1e12 if prof["launches"] else None
    traffic, _ = captured_traffic(min(args.chunk, ne)) if args.precision == "emu64" and b == 256 else (None, None)
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read+write, scaled from a 64-energy capture)",
                "achieved_counts": "algorithmic flops: 8 M N K per complex product (complex FP64-equivalent)",
                "pipe_achieved": pipe, "pipe_frac": (pipe / peak) if pipe else None,
                "pipe_flops_per_algorithmic": (prof["pipe_flops"] / prof["useful_flops"]) if prof["useful_flops"] else None,
                "kernel": kernel, "launches": prof["launches"], "avg_launch_ms": avg_ms,
                "algorithmic_flops_per_launch": prof["useful_flops"] / n_l,
                "share_of_step": prof["ms"] / ms if ms else None,
                "peak_source": f"{peak_src} ({'bf16 sustained' if bound == 'tensor' else 'cuBLAS/torch matmul on this GPU'})"}

    # ---------------------------------------------------------------- end to end (host buffers)
    e2e = None
    if not args.no_e2e:
        host = {k: v.cpu().pin_memory() for k, v in din.items()
                if isinstance(v, torch.Tensor)}
        hc = torch.empty_like(cur, device="cpu").pin_memory()
        hd = torch.empty_like(den, device="cpu").pin_memory()
        hci = torch.empty_like(cint, device="cpu").pin_memory()
        hdi = torch.empty_like(dint, device="cpu").pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = sum(t.numel() * t.element_size() for t in (hc, hd, hci, hdi))

        def e2e_step():
            for k, t in host.items():
                din[k].copy_(t, non_blocking=True)
            step()
            hc.copy_(cur, non_blocking=True)
            hd.copy_(den, non_blocking=True)
            hci.copy_(cint, non_blocking=True)
            hdi.copy_(dint, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(f0.elapsed_time(f1), ws)
        e2e = {"value": ws * ne * args.steps / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # ---------------------------------------------------------------- FP64 path on a subset
    fp64 = None
    if args.fp64_energies > 0 and args.precision != "fp64":
        nsub = min(args.fp64_energies, ne)
        idx = np.linspace(0, ne - 1, nsub).astype(int)
        Esub = dev["energies"][idx]
        p64 = q.Plan(q.make_desc(nb, b, "fp64", nsub, has_scattering=True,
                                 outputs=["current", "density"], offdiag_sigma=bt))
        din64 = q.upload(dev, Esub)
        c64 = torch.empty((nsub, nb - 1), dtype=torch.float64, device=cd)
        d64 = torch.empty((nsub, nb), dtype=torch.float64, device=cd)
        o64 = q.Outputs()
        o64.current, o64.density = c64.data_ptr(), d64.data_ptr()
        p64.solve(din64["_inputs"], o64, stream.cuda_stream)  # warm-up
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        p64.solve(din64["_inputs"], o64, stream.cuda_stream)
        g1.record(stream)
        torch.cuda.synchronize()
        t64 = g0.elapsed_time(g1) / 1e3
        c_h, d_h = cur[idx].cpu().numpy(), den[idx].cpu().numpy()
        c64n, d64n = c64.cpu().numpy(), d64.cpu().numpy()
        fp64 = {"value": ws * nsub / t64, "unit": UNIT, "energies_timed": int(nsub),
                "speedup_of_headline": value / (ws * nsub / t64),
                "headline_vs_fp64_gpu": {
                    "current": float(np.abs(c_h - c64n).max() / np.abs(c64n).max()),
                    "density": float(np.abs(d_h - d64n).max() / np.abs(d64n).max())}}
        del p64

    # ---------------------------------------------------------------- the other modes on the same workload
    # (all energies, same chunk and refinement; per-energy current and density kept for the errors)
    modes = {}
    if args.modes and args.precision == "emu64" and not args.no_modes:
        c_main, d_main = cur.cpu().numpy(), den.cpu().numpy()
        del plan, GR, GL
        torch.cuda.empty_cache()
        for m in args.modes.split(","):
            pm = q.Plan(q.make_desc(nb, b, m, min(args.chunk, ne), refine_max_iter=2, has_scattering=True,
                                    outputs=["current", "density"], offdiag_sigma=bt, refine_tol=args.refine_tol))
            cm = torch.empty_like(cur)
            dm = torch.empty_like(den)
            sm = torch.zeros_like(stat)
            om = q.Outputs()
            om.current, om.density, om.status_per_energy = cm.data_ptr(), dm.data_ptr(), sm.data_ptr()
            pm.solve(din["_inputs"], om, stream.cuda_stream)  # warm-up
            torch.cuda.synchronize()
            h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h0.record(stream)
            pm.solve(din["_inputs"], om, stream.cuda_stream)
            h1.record(stream)
            torch.cuda.synchronize()
            modes[m] = {"value": ws * ne / (h0.elapsed_time(h1) / 1e3), "unit": UNIT,
                        "status_ok": bool(torch.all(sm == 0).item()),
                        "_cur": cm.cpu().numpy(), "_den": dm.cpu().numpy()}
            pm.close()
            del pm
        cur_host, den_host = c_main, d_main
    else:
        cur_host, den_host = cur.cpu().numpy(), den.cpu().numpy()

    # ---------------------------------------------------------------- the strip and uneven workloads
    # (secondary single-GPU measurements, so that every benchmarked configuration appears in the one
    # line; rank 0 alone runs them, after every collective of the timed legs)
    others = {}
    if not args.no_others and args.precision == "emu64" and rank == 0:
        others = secondary_workloads(q, W)

    # ---------------------------------------------------------------- CPU oracle sample + error
    cpu = None
    err = None
    if rank == 0 and ws == 1:
        pool = list(np.linspace(0, ne - 1, 64).astype(int))
        rng = np.random.default_rng(7)
        rng.shuffle(pool)
        done, res, dt = cpu_oracle_sample(dev, args.cpu_seconds, pool)
        cpu = {"value": len(done) / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{len(done)} of the {ne} energies (numpy complex128, LAPACK inv, "
                         f"{dt:.1f} s)"}
        c_g, d_g = cur_host, den_host
        cr = np.stack([res[k][0] for k in done])
        dr = np.stack([res[k][1] for k in done])
        err = {"energies": len(done),
               "current": float(np.abs(c_g[done] - cr).max() / np.abs(cr).max()),
               "density": float(np.abs(d_g[done] - dr).max() / np.abs(dr).max())}
        for m, v in modes.items():
            v["error_vs_oracle"] = {"energies": len(done),
                                    "current": float(np.abs(v["_cur"][done] - cr).max() / np.abs(cr).max()),
                                    "density": float(np.abs(v["_den"][done] - dr).max() / np.abs(dr).max())}
    for v in modes.values():
        v.pop("_cur", None)
        v.pop("_den", None)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"emu64": "bf16-digits(tcgen05)+df32", "bf16x3": "bf16-digits(tcgen05)+df32",
                          "fp32": "c64", "fp64": "c128"}[args.precision],
                "data": "synthetic",
                "config": {"workload": f"random BT device b={b} N_B={nb} N_E={ne} on [-2,2], "
                                       + ("block-tridiagonal" if bt else "block-diagonal")
                                       + " scattering self-energies (seed 0)",
                           "global_batch": ne * ws, "precision": args.precision,
                           "energies_in_flight": min(args.chunk, ne),
                           "storage_bits": args.storage_bits,
                           "tc_stages": args.tc_stages, "tc_ctas": args.tc_ctas,
                           "refine_max_iter": 2, "refine_tol": args.refine_tol,
                           "plan_bytes_per_energy_in_flight": q.footprint(desc) // min(args.chunk, ne),
                           "l2": "inputs and working set (>= 16 GB) larger than L2; no flush"},
                "status_ok": status_ok,
                "gpu_launches": int(launches),
                "clocks": clocks, "roofline": roofline, "e2e": e2e, "fp64_path": fp64, "other_modes": modes,
                "other_workloads": others,
                "cpu_baseline": cpu, "error_vs_oracle": err}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
