"""Sharding of one sequence over ranks (the paper's parallel split, Sec. 1).

Rank r of `world` generates variates r*n .. (r+1)*n-1 of the same stream by
skip-ahead, so the shards need no exchange and their concatenation in rank
order is the single-stream sequence.  The only collective is the max of the
per-rank step times, taken for reporting.
"""
from __future__ import annotations


def shard_range(rank: int, world: int, n_per_rank: int) -> tuple[int, int]:
    """(offset, count) of rank `rank`'s block when every rank makes n_per_rank."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    return rank * n_per_rank, n_per_rank


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    if dist.get_backend() == "gloo":
        device = None  # gloo reduces host tensors
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
