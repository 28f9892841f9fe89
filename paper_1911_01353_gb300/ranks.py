"""Host-side helpers for running searches on several ranks.

Two ways to divide the work:

* independent spectra (DM trials): each rank takes a contiguous block of the
  items and searches them on its own GPU; ranks share no data, the results
  are merged on rank 0, and the only collective is the max over ranks of the
  timed duration;
* one spectrum split by template range (``search_split``): each rank
  searches a contiguous range of the bank's templates (its fundamentals'
  harmonic rows are made locally, also from templates outside the range);
  the stage max-projections are maxima over templates / fundamentals and the
  statistics are sums over them (Sec. 3), so one max-reduction per stage and
  one sum-reduction of the statistics give the whole search's result.
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


def template_range(n_templates: int, rank: int, world: int):
    """(t_lo, t_hi) of `rank` in a split of the bank by template index."""
    r = shard(n_templates, rank, world)
    return r.start, r.stop


def pack(values, t):
    """Packed max-projection entries (float bits << 32 | (0xFFFFFFFF - t)) as
    int64: the maximum of packed entries keeps the largest value and, on equal
    values, the lowest t (non-negative values only)."""
    import numpy as np
    v = np.asarray(values, dtype=np.float32)
    if np.any(v < 0):
        raise ValueError("packed max-projections hold non-negative powers")
    hi = v.view(np.uint32).astype(np.uint64) << np.uint64(32)
    lo = np.uint64(0xFFFFFFFF) - np.asarray(t).astype(np.uint64)
    return (hi | lo).view(np.int64)


def unpack(packed):
    """(float32 values, int64 t) of packed entries."""
    import numpy as np
    u = np.asarray(packed).view(np.uint64)
    return (u >> np.uint64(32)).astype(np.uint32).view(np.float32), \
        (np.uint64(0xFFFFFFFF) - (u & np.uint64(0xFFFFFFFF))).astype(np.int64)


def reduce_split(maxprojs, sums, dist=None):
    """In place over the ranks: element-wise MAX of every packed int64
    max-projection tensor and SUM of the statistics tensor (float64, any
    shape).  No-op on one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return
    for m in maxprojs:
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
    dist.all_reduce(sums, op=dist.ReduceOp.SUM)


def search_split(plan, spec, dist=None, stream=None):
    """One spectrum searched by all ranks of `dist` (one GPU each), split by
    template range: jerk_search_range on this rank's range, the reductions,
    then jerk_select.  Every rank returns the whole search's candidates."""
    import torch
    rank = dist.get_rank() if dist is not None and dist.is_initialized() else 0
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    lo, hi = template_range(int(plan.info.n_templates), rank, world)
    plan.search_range(spec, lo, hi, stream=stream)
    s1, s2, n = plan.range_sums()
    ns = int(plan.params.n_stages)
    sums = torch.tensor([s1, s2, n], dtype=torch.float64, device="cuda:%d" % plan.device)
    ms = [plan.maxproj_tensor(si) for si in range(ns)]
    reduce_split(ms, sums, dist)
    torch.cuda.synchronize(plan.device)
    s = sums.cpu().numpy()
    plan.select(s[0], s[1], s[2], stream=stream)
    return plan.candidates()
