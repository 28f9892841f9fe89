"""Tile-shape autotuner with a JSON cache.

The fused filter's tile shape has two free parameters: the segment (FFT)
length L, which fixes the transform size, the overlap wasted per segment and
the segments a CTA holds (two at L <= 4096, one at 8192), and the template
group size G, the number of templates one CTA walks with its segments
resident (its bank slice is shared by every CTA of the group through L2).
For a parameter set and a spectrum length every admissible (L, G) is timed
on the device with a noise spectrum, and the fastest is kept.  Results are
cached in a JSON file keyed by the search parameters and the length rounded
up to a power of two, so a later run reuses them.

Timing: CUDA events on the search's stream around jerk_search (the whole
path, enqueued without host synchronisation), median of `reps` searches
after one warm-up; everything goes through the library's C ABI.
"""
from __future__ import annotations

import json
import math
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "jerk_gb300_autotune.json")
SEG_LENS = (2048, 4096, 8192)
GROUP_SIZES = (0, 256, 512, 2048)         # 0: the library's own choice (32 MiB of bank)


def _key(zmax, dz, wmax, dw, stages, pad_bins, n_bins, seg_lens=SEG_LENS, group_sizes=GROUP_SIZES):
    bucket = 1 << max(10, math.ceil(math.log2(max(n_bins, 1))))
    return "z%d/%d w%d/%d s%s p%d n%d L%s G%s" % (zmax, dz, wmax, dw, "-".join(map(str, stages)), pad_bins, bucket,
                                                  "-".join(map(str, seg_lens)), "-".join(map(str, group_sizes)))


def load(path=DEFAULT_CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(cache, path=DEFAULT_CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_shape(zmax, dz, wmax, dw, stages, n_bins, seg_len, group_size=0, pad_bins=16, reps=3, device=0):
    """Median ms (CUDA events) of one search at this tile shape, or None when
    the shape is not admissible for the bank (or does not fit)."""
    import numpy as np
    import torch

    from . import jerk
    p = jerk.make_params(zmax, dz, wmax, dw, stages=stages, thresh=(1e30,) * len(stages),
                         pad_bins=pad_bins, seg_len=seg_len, max_bins=n_bins, max_candidates=1 << 16,
                         group_size=group_size)
    try:
        plan = jerk.Plan(p, device=device)
    except jerk.JerkError:
        return None
    try:
        rng = np.random.default_rng(0)
        spec = (rng.standard_normal(n_bins) + 1j * rng.standard_normal(n_bins)).astype(np.complex64)
        x = torch.from_numpy(spec).cuda(device)
        stream = torch.cuda.current_stream(device)
        plan.search(x, stream=stream)
        plan.candidates()
        ms = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.search(x, stream=stream)
            e1.record(stream)
            e1.synchronize()
            plan.candidates()
            ms.append(e0.elapsed_time(e1))
        return sorted(ms)[len(ms) // 2]
    finally:
        plan.close()


def time_seg_len(zmax, dz, wmax, dw, stages, n_bins, seg_len, pad_bins=16, reps=3, device=0):
    """time_shape at the library's own group size."""
    return time_shape(zmax, dz, wmax, dw, stages, n_bins, seg_len, 0, pad_bins, reps, device)


def best_shape(zmax, dz, wmax, dw, stages, n_bins, pad_bins=16, device=0, cache_path=DEFAULT_CACHE,
               seg_lens=SEG_LENS, group_sizes=GROUP_SIZES, refresh=False):
    """The fastest (segment length, group size) for this search (cached)."""
    cache = load(cache_path)
    key = _key(zmax, dz, wmax, dw, stages, pad_bins, n_bins, seg_lens, group_sizes)
    hit = cache.get(key)
    if not refresh and hit:
        return int(hit["seg_len"]), int(hit["group_size"])
    results = {}
    for L in seg_lens:
        for G in group_sizes:
            ms = time_shape(zmax, dz, wmax, dw, stages, n_bins, L, G, pad_bins, device=device)
            if ms is not None:
                results["%d/%d" % (L, G)] = ms
    if not results:
        raise RuntimeError("no admissible tile shape for %s" % key)
    best = min(results, key=results.get)
    L, G = (int(x) for x in best.split("/"))
    cache[key] = {"seg_len": L, "group_size": G, "ms": results}
    save(cache, cache_path)
    return L, G


def best_seg_len(zmax, dz, wmax, dw, stages, n_bins, pad_bins=16, device=0, cache_path=DEFAULT_CACHE,
                 candidates=SEG_LENS, refresh=False):
    """The fastest segment length at the library's own group size (cached)."""
    L, _ = best_shape(zmax, dz, wmax, dw, stages, n_bins, pad_bins, device, cache_path, candidates, (0,), refresh)
    return L
