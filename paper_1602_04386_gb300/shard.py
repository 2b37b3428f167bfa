"""Replica sharding across ranks (one process per GPU).

The graphs of the batched and serving forms are independent problems, so N
ranks split them with no data-path collective: rank r takes the graphs whose
global index is congruent to r modulo N, and the only communication is the
timing reduction at the end (the slowest rank's time, the total count).
Every rank holds its own plan on its own GPU.
"""
from __future__ import annotations

import os


def dist_env():
    """(world size, rank, local rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_indices(count: int, rank: int, world: int) -> list[int]:
    """Global indices of rank `rank` among `world` ranks (round robin, so
    that each rank's share of an ordered workload has the same size mix)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    return list(range(rank, count, world))


def reduce_max(value: float, dist=None, device=None) -> float:
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, dist=None, device=None) -> float:
    """Sum over the ranks (units processed by the whole job)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
