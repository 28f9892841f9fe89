"""Host-side helpers for running independent searches on several ranks.

The search partitions into independent problems (one spectrum per DM
trial), so ranks share no data: each rank takes a contiguous block of the
items, searches them on its own GPU, and the results are merged on rank 0.
The only collective is the max over ranks of the timed duration.
"""
from __future__ import annotations


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous block of item indices for `rank` (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def merge(per_rank):
    """Merge per-rank lists of (item, stage, p, t, power) records into one
    list sorted by (item, stage, p)."""
    out = [rec for recs in per_rank for rec in recs]
    out.sort(key=lambda r: (r[0], r[1], r[2]))
    return out


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the job's wall time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])
