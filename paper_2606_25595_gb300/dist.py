"""Energy-parallel execution across ranks (one process per GPU), host side only.

Energies are independent (Sec. II-A: Eq. 2 is solved separately at every energy), so the solve
shards with no exchange inside it.  Energies are dealt round-robin rather than in contiguous
blocks, because the cost of an energy varies along the grid (refinement sweeps, decimation sweeps
near band edges) and neighbouring energies cost alike.  The one combine is the sum of the
energy-integrated current and density vectors (N_B - 1 and N_B doubles), after each rank has
integrated its own energies with the weights of the full grid.

Works with any torch.distributed backend: gloo on CPU tensors, NCCL on CUDA tensors.
"""
from __future__ import annotations

import os

import numpy as np

__all__ = ["init", "shard", "barrier", "max_over_ranks", "reduce_integrals"]


def init(backend: str | None = None):
    """(rank, world_size, local_rank) from the torchrun environment; initialises the process group
    when WORLD_SIZE > 1 (NCCL when CUDA is available, else gloo)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(lr)
    if not dist.is_initialized():
        dist.init_process_group(backend)
    return dist.get_rank(), ws, lr


def shard(n_energies: int, rank: int, world: int) -> np.ndarray:
    """Indices of the energies this rank solves: rank, rank + world, ..."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return np.arange(rank, n_energies, world)


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _device():
    import torch
    import torch.distributed as dist
    return torch.device("cuda") if dist.get_backend() == "nccl" else torch.device("cpu")


def max_over_ranks(x: float, world: int) -> float:
    """The largest x over all ranks (timing: the job ends with its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_integrals(current_int: np.ndarray, density_int: np.ndarray, world: int):
    """Sum the per-rank partial energy integrals (each rank integrated its shard with the full
    grid's weights); returns the totals on every rank."""
    if world <= 1:
        return np.asarray(current_int, dtype=np.float64), np.asarray(density_int, dtype=np.float64)
    import torch
    import torch.distributed as dist
    nc = len(current_int)
    t = torch.tensor(np.concatenate([np.asarray(current_int, np.float64), np.asarray(density_int, np.float64)]),
                     dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    a = t.cpu().numpy()
    return a[:nc], a[nc:]
