"""Query sharding across GPUs (one process per GPU, replicas only).

Queries of a batch are independent, so the online phase shards by query with
no exchange on the data path: every rank holds the same basis and solves a
contiguous slice of the parameter vectors.  The only collective is the
max-over-ranks of the step time used for reporting.
"""
from __future__ import annotations


def shard_range(n_total: int, rank: int, world: int):
    """Contiguous, balanced slice [start, stop) of n_total queries for `rank` of `world`."""
    if world < 1 or not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of `value` over the ranks of the default process group (identity without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
