"""The failure path of the bounded device waits, on the GPU, without a fault.

jerk_check_waits makes one GPU thread wait, with the bounded wait the filter
kernels use, on a barrier phase that nothing completes.  The wait must give
up after its limit, the plan must report JERK_ETIMEOUT, and the plan and its
CUDA context must stay usable: the same search before and after gives the
same candidates.  The debug build's test hook (jerk_check_inject) then makes
the filter kernels' own waits expire, one kind at a time, inside a search.
"""
import json
import os
import subprocess
import sys
import time

import numpy as np
import pytest

import oracle
import synth
from parity import jerk_params, lib_ready

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib_ready()


def test_expired_wait_is_reported_and_the_plan_recovers(pkg):
    from paper_1911_01353_gb300 import jerk
    F = synth.spectrum(30000, 41, [synth.Signal(9000.5, 4.0, 20.0, 40.0, 0.2)])
    op = oracle.Params(12, 2, 40, 20, stages=(1, 2), thresh=(12.0, 17.0))
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        x = torch.from_numpy(F).cuda()
        plan.search(x)
        before = [(c.stage, c.p, c.t, c.power) for c in plan.candidates()]
        t0 = time.perf_counter()
        assert plan.check_waits(20000) == jerk.JERK_ETIMEOUT          # 20 ms limit
        assert time.perf_counter() - t0 >= 0.02
        for limit in (1, 500):                                         # repeatable
            assert plan.check_waits(limit) == jerk.JERK_ETIMEOUT
        plan.search(x)
        after = [(c.stage, c.p, c.t, c.power) for c in plan.candidates()]
        with pytest.raises(jerk.JerkError) as e:
            plan.check_waits(0)
        assert e.value.code == jerk.JERK_EINVAL
    assert after == before and len(before) > 0


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _inject_run(checks):
    env = dict(os.environ)
    env["JERK_CHECKS"] = "1" if checks else "0"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "inject_run.py")], capture_output=True,
                       text=True, timeout=900, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_filter_waits_expire_and_the_plan_recovers():
    """Inside a search, with no fault: a template copy left out (FP32 and
    tensor-core filters) and a tensor-core product's completion left out (each
    product) make the kernels' bounded waits expire; the search reports
    JERK_ETIMEOUT after about the one-second limit, and the same plan then
    gives the clean search's candidates again.  The release build refuses the
    hook."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_01353_gb300 import jerk
    out = _inject_run(True)
    assert out["checks"]
    seen = set()
    for r in out["runs"]:
        assert r["inject"] == jerk.JERK_OK, r
        assert r["status"] == jerk.JERK_ETIMEOUT, r
        assert 0.5 <= r["seconds"] < 60.0, r
        assert r["recovered"] and r["candidates"] > 0, r
        seen.add((r["precision"], r["mode"]))
    assert seen == {(0, 1), (2, 1), (2, 2), (2, 3)}
    rel = _inject_run(False)
    assert not rel["checks"]
    assert [r["inject"] for r in rel["runs"]] == [jerk.JERK_ESTATE, jerk.JERK_ESTATE]
