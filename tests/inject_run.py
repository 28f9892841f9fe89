"""Helper of test_gpu_failure.py (not a test module): with the debug build's
test hook (jerk_check_inject), make each bounded wait of the filter kernels
expire once -- the template copy (both filters), the completion of either
tensor-core product -- and print, as one JSON line, what each search returned,
how long it took, and whether the same plan then gave the clean search's
candidates again.  Run with JERK_CHECKS=1 it uses the debug build; with
JERK_CHECKS=0 it only reports the release build's answer to the hook."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import synth  # noqa: E402
from paper_1911_01353_gb300 import build, jerk  # noqa: E402


def key(cands):
    return sorted((int(c.stage), int(c.p), int(c.t)) for c in cands)


def main():
    checks = os.environ.get("JERK_CHECKS") == "1"
    if checks:
        build.build(checks=True)
    else:
        build.build()
    n = 30000
    F = synth.spectrum(n, 41, [synth.Signal(9000.5, 4.0, 20.0, 40.0, 0.2)])
    out = {"checks": checks, "runs": []}
    for prec in (0, 2):
        p = jerk.make_params(12, 2, 40, 20, stages=(1, 2), thresh=(12.0, 17.0), max_bins=n, precision=prec)
        with jerk.Plan(p) as plan:
            x = torch.from_numpy(F).cuda()
            plan.search(x)
            clean = key(plan.candidates())
            if not checks:
                out["runs"].append({"precision": prec, "inject": plan.check_inject(1, 3)})
                continue
            for mode in ((1,) if prec == 0 else (1, 2, 3)):
                code = plan.check_inject(mode, 3)
                t0 = time.perf_counter()
                plan.search(x)
                try:
                    plan.candidates()
                    status = jerk.JERK_OK
                except jerk.JerkError as e:
                    status = e.code
                dt = time.perf_counter() - t0
                plan.check_inject(0)
                plan.search(x)
                again = key(plan.candidates())
                out["runs"].append({"precision": prec, "mode": mode, "inject": code, "status": status,
                                    "seconds": dt, "recovered": again == clean, "candidates": len(clean)})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
