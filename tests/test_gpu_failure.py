"""The failure path of the bounded device waits, on the GPU, without a fault.

jerk_check_waits makes one GPU thread wait, with the bounded wait the filter
kernels use, on a barrier phase that nothing completes.  The wait must give
up after its limit, the plan must report JERK_ETIMEOUT, and the plan and its
CUDA context must stay usable: the same search before and after gives the
same candidates.
"""
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
