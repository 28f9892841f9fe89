"""Writes the stored oracle results under tests/golden/.

Calls only ``oracle`` and ``synth`` (never the CUDA path).  Run from the
repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402


def small_single():
    wl = synth.small_single()
    p = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=wl.stages, thresh=wl.thresh)
    res = oracle.search(wl.make(), p)
    return {
        "workload": wl.name,
        "params": {"zmax": p.zmax, "dz": p.dz, "wmax": p.wmax, "dw": p.dw,
                   "numbetween": p.numbetween, "pad_bins": p.pad_bins,
                   "stages": list(p.stages), "thresh_mode": p.thresh_mode,
                   "thresh": list(p.thresh), "norm_block": p.norm_block},
        "candidates": [list(c) for c in res.candidates],
        "stats": {str(h): list(v) for h, v in res.stats.items()},
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "small_single_candidates.json")
    with open(out, "w") as f:
        json.dump(small_single(), f, indent=1)
        f.write("\n")
    print("wrote", out)
