"""GPU parity of the configurations the benchmark times, each run exactly as it is timed and
compared with the FP64 oracle at sampled energies.

* the batched mixed-precision device (b = 256, N_B = 64, 512 energies on [-2, 2]) in the emulated-FP64
  mode with all 512 energies in flight and adaptive refinement at tol = 2^-12;
* an uneven batch of eight devices of different (N_B, b) replayed from one CUDA graph, equal bit for
  bit to the same solves launched directly, and within each mode's bar of the oracle;
* the paper's NR-L block shape (b = 3408, N_B = 10, Sec. V) with per-energy self-energies streamed
  from host memory.
Bars: current and density within 1e-6 of the oracle (max over the sampled energies of |x - x_ref|,
relative to max |x_ref|), the emulated mode's G blocks within 1e-7 (relative Frobenius, per energy).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

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


def _obs_err(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def _blk_err(got, ref):
    return max(float(np.linalg.norm(got[e] - ref[e]) / np.linalg.norm(ref[e])) for e in range(ref.shape[0]))


def test_mixed_workload_as_benchmarked(q):
    """b = 256, N_B = 64, 512 energies, emulated FP64, all 512 energies in one chunk, refinement
    until ||I - A X||_F <= 2^-12 (at most 2 sweeps), the benchmark's outputs; 8 energies spread over
    [-2, 2] against the oracle.  The energy integrals are checked against the trapezoid rule applied
    to the same solve's per-energy values."""
    import torch
    cfg = W.MIXED_CFG
    nb, b, ne = cfg["n_blocks"], cfg["b"], cfg["n_energies"]
    dev = W.random_device(b, nb, n_energies=ne, seed=0)
    din = q.upload(dev)
    outs = ["GR_diag", "GL_diag", "current", "density", "integrals"]
    plan = q.Plan(q.make_desc(nb, b, "emu64", ne, refine_max_iter=2, has_scattering=True, outputs=outs,
                              refine_tol=2.0 ** -12))
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
    plan.solve(din["_inputs"], o, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert bool(torch.all(stat == 0))
    idx = np.linspace(0, ne - 1, 8).astype(int)
    ref = O.solve(dev, energy_indices=idx, keep_blocks=True)
    c, d = cur.cpu().numpy(), den.cpu().numpy()
    assert _obs_err(c[idx], ref["current"]) < 1e-6
    assert _obs_err(d[idx], ref["density"]) < 1e-6
    ti = torch.as_tensor(idx, device=cd)
    assert _blk_err(GR.index_select(0, ti).cpu().numpy(), ref["GR_diag"]) < 1e-7
    assert _blk_err(GL.index_select(0, ti).cpu().numpy(), ref["GL_diag"]) < 1e-7
    w = W.trapezoid_weights(dev["energies"])
    assert np.abs(cint.cpu().numpy() - w @ c).max() < 1e-12 * np.abs(w @ c).max()
    assert np.abs(dint.cpu().numpy() - (w @ d) / (2 * np.pi)).max() < 1e-12 * np.abs(w @ d).max()
    plan.close()


@pytest.mark.parametrize("precision", ["emu64", "fp32"])
def test_uneven_batch_graph_replay(q, precision):
    """Eight devices of the uneven workload's shapes scaled by 1/4 (b in 32..128, N_B in 4..32), six
    energies each, two energies in flight: the CUDA-graph replay equals direct launches bit for bit;
    the emulated-FP64 results are within 1e-6 (current, density) of the oracle, the FP32 ones within
    the FP32 mode's bar (density 1e-4, G^R diagonal blocks 5e-4)."""
    from paper_2606_25595_gb300.batch import UnevenBatch
    devs = W.uneven_batch(n_energies=6, scale=0.25)
    outs = ("GR_diag", "current", "density", "integrals")
    ub = UnevenBatch(devs, precision, chunks=[2] * len(devs), outputs=outs)
    ub.launch()
    eager = ub.results()
    ub.capture()
    for _ in range(2):
        ub.replay()
    replay = ub.results()
    for e, r in zip(eager, replay):
        assert np.all(e["status"] == 0)
        for k in e:
            assert np.array_equal(e[k], r[k]), k
    for dev, r in zip(devs, replay):
        idx = [0, 5]
        ref = O.solve(dev, energy_indices=idx, keep_blocks=True)
        if precision == "emu64":
            assert _obs_err(r["current"][idx], ref["current"]) < 1e-6
            assert _obs_err(r["density"][idx], ref["density"]) < 1e-6
            assert _blk_err(r["GR_diag"][idx], ref["GR_diag"]) < 1e-7
        else:
            assert _obs_err(r["density"][idx], ref["density"]) < 1e-4
            assert _blk_err(r["GR_diag"][idx], ref["GR_diag"]) < 5e-4
    ub.close()


@pytest.mark.parametrize("precision", ["emu64", "fp32"])
def test_group_solve_equals_solo_solves(q, precision):
    """A group solve of the eight scaled uneven devices (each device on its own stream and host
    thread) equals the same plans solved one by one, bit for bit, without pooling (the default) and
    with the tensor-core products pooled into shared persistent launches at a two-wave threshold,
    where its pooled launches cover more products than there are launches."""
    from paper_2606_25595_gb300.batch import UnevenBatch
    devs = W.uneven_batch(n_energies=4, scale=0.25)
    outs = ("GR_diag", "GL_diag", "current", "density", "integrals")
    solo = UnevenBatch(devs, precision, chunks=[2] * len(devs), outputs=outs, grouped=False)
    solo.launch()
    r_solo = solo.results()
    solo.close()
    grp = UnevenBatch(devs, precision, chunks=[2] * len(devs), outputs=outs, grouped=True)
    grp.launch()
    r_grp = grp.results()
    assert grp.group.launches() == 0
    grp.group.set_pool_waves(2)
    grp.launch()
    r_pool = grp.results()
    for a, b, c in zip(r_solo, r_grp, r_pool):
        assert np.all(a["status"] == 0)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
            assert np.array_equal(a[k], c[k]), k
    assert 0 < grp.group.launches() < grp.group.pooled_products()
    grp.close()


@pytest.mark.parametrize("precision,stages", [("emu64", 2), ("fp32", 2), ("bf16x3", 4)])
def test_schedule_knobs_leave_results_unchanged(q, precision, stages):
    """The product kernel's schedule (pipeline stages, persistent CTAs per launch) and the group's
    pooling threshold change only the order tiles are taken in, never a tile's arithmetic: the scaled
    uneven devices solved with the non-default stage count and 37 CTAs per launch, and as a group at
    every pooling threshold the autotuner searches, equal the default schedule bit for bit."""
    from paper_2606_25595_gb300 import autotune
    from paper_2606_25595_gb300.batch import UnevenBatch
    devs = W.uneven_batch(n_energies=4, scale=0.25)
    outs = ("GR_diag", "GL_diag", "current", "density")
    n = len(devs)
    ref = UnevenBatch(devs, precision, chunks=[2] * n, outputs=outs, grouped=False)
    ref.launch()
    r_ref = ref.results()
    ref.close()
    alt = UnevenBatch(devs, precision, chunks=[2] * n, outputs=outs, grouped=False,
                      stages=[stages] * n, ctas=[37] * n)
    alt.launch()
    r_alt = alt.results()
    alt.close()
    for a, b in zip(r_ref, r_alt):
        assert np.all(a["status"] == 0)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    grp = UnevenBatch(devs, precision, chunks=[2] * n, outputs=outs, grouped=True, stages=[stages] * n)
    for w in (0, 1, 2, 4):
        grp.group.set_pool_waves(w)
        grp.launch()
        for a, b in zip(r_ref, grp.results()):
            for k in a:
                assert np.array_equal(a[k], b[k]), (w, k)
    best = autotune.best_pool_waves(grp, refresh=True)
    assert best in (0, 1, 2, 4)
    grp.close()
    assert stages in autotune.STAGE_CHOICES[precision]


@pytest.mark.slow
def test_nrl_shape_streamed_sigma(q):
    """The paper's NR-L block shape, b = 3408 and N_B = 10 (Sec. V; split-K products with seven
    digits, six levels of recursive inverse), per-energy self-energies streamed from pinned host
    memory slice by slice, one energy: emulated-FP64 current and density within 1e-6 of the oracle,
    G blocks within 1e-7."""
    cfg = W.NRL_CFG
    # two energies of self-energies (so they are per energy); the first one is solved
    dev = W.nrl_device(cfg["b"], cfg["n_blocks"], n_energies=2, e_lo=0.37, e_hi=0.55)
    res = q.solve_device(dev, "emu64", outputs=["GR_diag", "GL_diag", "current", "density"],
                         energies=dev["energies"][:1], max_energies_in_flight=1, sigma_stream=True)
    assert np.all(res["status"] == 0)
    ref = O.solve(dev, energy_indices=[0], keep_blocks=True)
    assert _obs_err(res["current"], ref["current"]) < 1e-6
    assert _obs_err(res["density"], ref["density"]) < 1e-6
    assert _blk_err(res["GR_diag"][0], ref["GR_diag"][0]) < 1e-7
    assert _blk_err(res["GL_diag"][0], ref["GL_diag"][0]) < 1e-7
