"""Multi-process plumbing around the projector (one process per GPU).

Two ways to use several GPUs, both without any collective inside F:

* replicas (what the benchmark runs): every rank projects its own copy of the
  workload; the job's throughput is the units all ranks processed divided by
  the slowest rank's time (`max_over_ranks`);
* view sharding: the rays of one problem are split into contiguous blocks
  (`shard`), each rank projects its block, and F^T of the whole problem is
  the sum of the ranks' partial back-projections (`sum_partials`, the one
  exchange step: an all-reduce of the volume).

Everything here is host logic on torch.distributed; it runs under NCCL on
GPUs and under gloo on CPU tensors alike.
"""
from __future__ import annotations

import os

import torch


def rank_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n: int, rank: int, world: int):
    """Contiguous block [lo, hi) of n items for `rank`; blocks differ in size
    by at most one and cover 0..n-1 exactly once."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks (the slowest rank's time); the value
    itself when torch.distributed is not initialised."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput of replicas: all ranks' units over the slowest time."""
    if seconds <= 0:
        raise ValueError("seconds must be positive")
    return world * units_per_rank / seconds


def sum_partials(volume: torch.Tensor) -> torch.Tensor:
    """In place: the sum over ranks of each rank's partial back-projection
    (F^T of a view-sharded problem). Identity on a single rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(volume, op=dist.ReduceOp.SUM)
    return volume
