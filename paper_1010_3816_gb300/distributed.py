"""Multi-GPU helpers: one process per GPU, no data-path collective.

A single solve is not split across GPUs (its r*-slab decomposition would need
one halo exchange per Lax-Wendroff step; not built).  Independent solves --
the instances of a batch, or replicas of one workload -- are sharded across
ranks, and only timings cross process boundaries.
"""
from __future__ import annotations

from typing import List, Sequence


def shard(costs: Sequence[float], rank: int, world: int) -> List[int]:
    """Indices of the items rank `rank` runs: longest-processing-time-first
    assignment of items with the given costs to `world` ranks (greedy, ties
    to the lowest rank), returned in increasing order.  Every item goes to
    exactly one rank; the same on every rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    load = [0.0] * world
    owner = [0] * len(costs)
    for k in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += costs[k]
    return [k for k in range(len(costs)) if owner[k] == rank]


def reduce_max(value: float, device=None) -> float:
    """Max of a float over all ranks of the default process group (identity
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
