"""Segment-length autotuner with a JSON cache.

For a parameter set and a spectrum length, every admissible segment (FFT)
length L is timed on the device with a noise spectrum, and the fastest is
kept.  Results are cached in a JSON file keyed by the search parameters and
the length rounded up to a power of two, so a later run reuses them.

All timing goes through the library's C ABI (jerk_search + jerk_candidates).
"""
from __future__ import annotations

import json
import math
import os
import time

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "jerk_gb300_autotune.json")
CANDIDATES = (2048, 4096, 8192)


def _key(zmax, dz, wmax, dw, stages, pad_bins, n_bins):
    bucket = 1 << max(10, math.ceil(math.log2(max(n_bins, 1))))
    return "z%d/%d w%d/%d s%s p%d n%d" % (zmax, dz, wmax, dw, "-".join(map(str, stages)), pad_bins, bucket)


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


def time_seg_len(zmax, dz, wmax, dw, stages, n_bins, seg_len, pad_bins=16, reps=3, device=0):
    """Median ms of one search (jerk_search + jerk_candidates) at this L, or
    None when L is not admissible for the bank."""
    import numpy as np
    import torch

    from . import jerk
    p = jerk.make_params(zmax, dz, wmax, dw, stages=stages, thresh=(1e30,) * len(stages),
                         pad_bins=pad_bins, seg_len=seg_len, max_bins=n_bins, max_candidates=1 << 16)
    try:
        plan = jerk.Plan(p, device=device)
    except jerk.JerkError:
        return None
    try:
        rng = np.random.default_rng(0)
        spec = (rng.standard_normal(n_bins) + 1j * rng.standard_normal(n_bins)).astype(np.complex64)
        x = torch.from_numpy(spec).cuda(device)
        plan.search(x)
        plan.candidates()
        ms = []
        for _ in range(reps):
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            plan.search(x)
            plan.candidates()
            ms.append(1e3 * (time.perf_counter() - t0))
        return sorted(ms)[len(ms) // 2]
    finally:
        plan.close()


def best_seg_len(zmax, dz, wmax, dw, stages, n_bins, pad_bins=16, device=0, cache_path=DEFAULT_CACHE,
                 candidates=CANDIDATES, refresh=False):
    """The fastest segment length for this search (cached)."""
    cache = load(cache_path)
    key = _key(zmax, dz, wmax, dw, stages, pad_bins, n_bins)
    if not refresh and key in cache:
        return int(cache[key]["seg_len"])
    results = {}
    for L in candidates:
        ms = time_seg_len(zmax, dz, wmax, dw, stages, n_bins, L, pad_bins, device=device)
        if ms is not None:
            results[str(L)] = ms
    if not results:
        raise RuntimeError("no admissible segment length for %s" % key)
    best = min(results, key=results.get)
    cache[key] = {"seg_len": int(best), "ms": results}
    save(cache, cache_path)
    return int(best)
