"""Serving loop: results are the same alone, in the mix and in a merged batch; prefix solves match the
oracle; requests that can never fit the HBM budget are refused."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2606_25595_gb300 import build
    build.build()
    from paper_2606_25595_gb300 import serve
    devs = {"b64": W.random_device(64, 16, n_energies=4, seed=61),
            "b128": W.random_device(128, 12, n_energies=4, seed=62)}
    models = {k: serve.DeviceModel(d, k) for k, d in devs.items()}
    return serve, devs, models


def _requests(serve):
    E = np.linspace(-1.5, 1.5, 9)
    return [serve.Request(0, "b64", 16, E[:7], "emu64", 0.1, -0.1, 0.0),
            serve.Request(1, "b128", 9, E[2:], "fp32", 0.0, 0.0, 0.0),
            serve.Request(2, "b64", 11, E[::2], "fp32", 0.2, 0.0, 0.0005),
            serve.Request(3, "b128", 12, E[:5], "emu64", 0.0, 0.0, 0.001)]


def test_results_identical_alone_and_in_the_mix(env):
    """Each request solved alone (one slot, one request at a time) and in an overlapping mix (three
    slots, staggered arrivals) gives bitwise-identical current and density: the plans are
    independent workspaces and every kernel is deterministic."""
    serve, devs, models = env
    alone = {}
    for r in _requests(serve):
        srv = serve.Server(models, slots=1)
        r.t_arrival = 0.0
        srv.run([r])
        alone[r.rid] = r.result
    srv = serve.Server(models, slots=3)
    reqs = _requests(serve)
    stats = srv.run(reqs)
    assert stats["completed"] == len(reqs)
    for r in reqs:
        assert np.all(r.result["status"] == 0)
        for k in ("current", "density", "current_int", "density_int"):
            assert np.array_equal(r.result[k], alone[r.rid][k]), (r.rid, k)


def test_merged_batch_equals_solo_runs(env):
    """Four requests queued together on one slot run as one merged batch (a group solve: their small
    products share persistent launches), and each one's current, density and integrals equal its solo
    run bit for bit."""
    serve, devs, models = env
    alone = {}
    for r in _requests(serve):
        srv = serve.Server(models, slots=1, group_size=1)
        r.t_arrival = 0.0
        srv.run([r])
        alone[r.rid] = r.result
    srv = serve.Server(models, slots=1, group_size=4)
    reqs = _requests(serve)
    for r in reqs:
        r.t_arrival = 0.0
    stats = srv.run(reqs)
    assert stats["completed"] == 4 and stats["largest_batch"] == 4 and stats["batches"] == 1, stats
    for r in reqs:
        assert np.all(r.result["status"] == 0)
        for k in ("current", "density", "current_int", "density_int"):
            assert np.array_equal(r.result[k], alone[r.rid][k]), (r.rid, k)


def test_request_beyond_the_budget_is_refused(env):
    """A request whose plan footprint exceeds the HBM budget is refused at submit with a reason;
    the others complete."""
    serve, devs, models = env
    from paper_2606_25595_gb300 import footprint, make_desc
    small = footprint(make_desc(16, 64, "fp32", 128, 2, has_scattering=True,
                                outputs=["current", "density", "integrals"]))
    srv = serve.Server(models, slots=2, hbm_budget=small + 1)
    reqs = [serve.Request(0, "b64", 16, np.linspace(-1, 1, 5), "fp32", 0.0, 0.0, 0.0),
            serve.Request(1, "b128", 12, np.linspace(-1, 1, 5), "emu64", 0.0, 0.0, 0.0)]
    stats = srv.run(reqs, time_limit=60.0)
    assert stats["completed"] == 1 and stats["rejected"] == 1, stats
    assert "rejected" in reqs[1].result and np.all(reqs[0].result["status"] == 0)


def test_prefix_solve_matches_oracle(env):
    """A plan sized for the model's 12 slices solving its first 9 (inputs.n_blocks) equals the
    oracle on the 9-slice device."""
    serve, devs, models = env
    d = devs["b128"]
    sub = dict(d)
    nb = 9
    sub["n_blocks"] = nb
    sub["H_diag"] = d["H_diag"][:nb]
    sub["H_upper"] = d["H_upper"][:nb - 1]
    sub["SigR"] = d["SigR"][:, :nb]
    sub["SigL"] = d["SigL"][:, :nb]
    E = np.linspace(-1.0, 1.0, 3)
    sub["energies"] = E
    ref = O.solve(sub, keep_blocks=False)
    srv = serve.Server(models, slots=1)
    r = serve.Request(0, "b128", nb, E, "emu64", 0.0, 0.0, 0.0)
    srv.run([r])
    for k in ("current", "density"):
        err = np.abs(r.result[k] - ref[k]).max() / np.abs(ref[k]).max()
        assert err < 1e-6, (k, err)
