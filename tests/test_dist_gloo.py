"""The multi-rank path on CPU: two gloo ranks each solve a round-robin shard of the energy grid (with
the oracle, since there is no GPU here), integrate it with the full grid's weights, and the sum of
the partial integrals over ranks equals the single-process integral; the slowest-rank timing reduce
returns the maximum."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _device():
    import workloads as W
    return W.strip(W=4, n_blocks=5, n_energies=15, eta=1e-3, seed=3)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as tdist

    import oracle as O
    from paper_2606_25595_gb300 import dist as D
    try:
        r, ws, _ = D.init("gloo")
        dev = _device()
        idx = D.shard(dev["energies"].size, r, ws)
        part = O.solve(dev, energy_indices=idx, keep_blocks=False)
        ci, di = D.reduce_integrals(part["current_int"], part["density_int"], ws)
        t = D.max_over_ranks(0.5 + r, ws)
        D.barrier(ws)
        q.put((r, idx.tolist(), ci, di, t))
        tdist.destroy_process_group()
    except Exception as exc:  # report instead of hanging the parent
        q.put((rank, "error", repr(exc), None, None))


def test_two_rank_energy_sharding_gloo():
    import multiprocessing as mp

    import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(2):
            r, idx, ci, di, t = q.get(timeout=180)
            assert idx != "error", ci
            got[r] = (idx, ci, di, t)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    dev = _device()
    full = O.solve(dev, keep_blocks=False)
    # the shards are disjoint and cover the grid, round-robin
    assert got[0][0] == list(range(0, 15, 2)) and got[1][0] == list(range(1, 15, 2))
    for r in (0, 1):
        _, ci, di, t = got[r]
        assert np.allclose(ci, full["current_int"], rtol=1e-12, atol=1e-15)
        assert np.allclose(di, full["density_int"], rtol=1e-12, atol=1e-15)
        assert t == 1.5


def test_shard_single_rank_and_bounds():
    from paper_2606_25595_gb300 import dist as D
    assert D.shard(5, 0, 1).tolist() == [0, 1, 2, 3, 4]
    with pytest.raises(ValueError):
        D.shard(5, 2, 2)
    ci, di = D.reduce_integrals([1.0], [2.0, 3.0], 1)
    assert ci.tolist() == [1.0] and di.tolist() == [2.0, 3.0]
