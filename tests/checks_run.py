"""Helper of test_gpu_checks.py (not a test module): run a fixed set of
searches (single, batched, sub-grid, split by template range) and plane rows
through the library loaded by the binding and print, as one JSON
line, their candidates and the plan's bounds-check counters.  Run with
JERK_CHECKS=1 it uses the debug build, whose kernels check the indices of
their global stores and copies."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import synth  # noqa: E402
from paper_1911_01353_gb300 import build, jerk  # noqa: E402


def key(cands):
    return sorted((int(c.item), int(c.stage), int(c.p), int(c.t)) for c in cands)


def main():
    if os.environ.get("JERK_CHECKS") == "1":
        build.build(checks=True)
    else:
        build.build()
    out = {"runs": {}, "checks": []}
    n = 1 << 15
    F = synth.spectrum(n, 31, [synth.Signal(3000.0, 2.0, 20.0, 6.0, 0.4)], harmonics=8)
    G = synth.spectrum(20001, 32, [synth.Signal(4000.5, -4.0, 0.0, 30.0, 0.1)], harmonics=4)
    for prec in (0, 2):
        p = jerk.make_params(16, 2, 160, 20, stages=(1, 2, 4, 8), thresh=(12.0, 18.0, 26.0, 40.0),
                             max_bins=n + 20001, precision=prec, max_batch=2)
        with jerk.Plan(p) as plan:
            plan.search(torch.from_numpy(F).cuda())
            out["runs"]["search%d" % prec] = key(plan.candidates())
            plan.search_batch([torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda()])
            out["runs"]["batch%d" % prec] = key(plan.candidates())
            plan.search_batch([torch.from_numpy(G).cuda()], zmax=[8], wmax=[60])
            out["runs"]["grid%d" % prec] = key(plan.candidates())
            # one search split in two template ranges, merged (as ranks would merge it)
            x = torch.from_numpy(F).cuda()
            T = plan.info.n_templates
            merged, tot = None, np.zeros((3, 4))
            for lo, hi in ((0, T // 2), (T // 2, T)):
                plan.search_range(x, lo, hi)
                tot += np.stack(plan.range_sums())
                parts = [plan.maxproj_tensor(si).clone() for si in range(4)]
                merged = parts if merged is None else [torch.maximum(a, b) for a, b in zip(merged, parts)]
            for si in range(4):
                plan.maxproj_tensor(si).copy_(merged[si])
            torch.cuda.synchronize()
            plan.select(tot[0], tot[1], tot[2])
            out["runs"]["split%d" % prec] = key(plan.candidates())
            rows = torch.empty((3, 2 * n), dtype=torch.float32, device="cuda")
            plan.plane(torch.from_numpy(F).cuda(), 10, 3, rows)
            r = rows.cpu().numpy()
            out["runs"]["plane%d" % prec] = [float(np.max(r)), float(np.sum(r, dtype=np.float64))]
            v, site, on = plan.check_counts()
            out["checks"].append({"precision": prec, "violations": v, "first_site": site, "enabled": on})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
