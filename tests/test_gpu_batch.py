"""Batched search of uneven-length spectra (DM trials) through the C ABI.

Every spectrum of a batch must give exactly what it gives alone (same cells,
templates, FP32 powers and statistics), with and without CUDA-graph replay,
and a replay with new input buffers must follow the new data.  One spectrum
is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import PLANE_TOL, compare_candidates, jerk_params, lib_ready

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LENGTHS = (30000, 17777, 50001, 1025, 8192)


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib_ready()


@pytest.fixture(scope="module")
def spectra():
    out = []
    for i, n in enumerate(LENGTHS):
        sig = [synth.Signal(n / 3 + 0.25 * i, 4.0 - 2 * i, 20.0 * (i % 3 - 1), 30.0 + i, 0.3 * i)]
        out.append(synth.spectrum(n, 300 + i, sig, harmonics=2))
    return out


def _params(mode="abs"):
    return oracle.Params(12, 2, 40, 20, stages=(1, 2, 4), thresh_mode=mode,
                         thresh=(12.0, 17.0, 24.0) if mode == "abs" else (6.0, 6.0, 6.0))


def _key(c):
    return (int(c.item), int(c.stage), int(c.p), int(c.t), float(c.power))


def _alone(pkg, plan, specs):
    got = []
    stats = []
    for F in specs:
        plan.search(torch.from_numpy(F).cuda())
        got.append([_key(c) for c in plan.candidates()])
        stats.append(plan.stats(0))
    return got, stats


@pytest.mark.parametrize("mode", ["abs", "sigma"])
def test_batch_equals_alone(pkg, spectra, mode):
    op = _params(mode)
    p = jerk_params(op, sum(LENGTHS))
    p.max_batch = len(LENGTHS)
    with pkg.Plan(p) as plan:
        alone, stats_alone = _alone(pkg, plan, spectra)
        dev = [torch.from_numpy(F).cuda() for F in spectra]
        for graph in (False, True, True):             # the second graph call is a replay
            plan.search_batch(dev, graph=graph)
            cands = plan.candidates()
            for i in range(len(spectra)):
                mine = [(0,) + _key(c)[1:] for c in cands if c.item == i]
                assert mine == alone[i], (graph, i)
                assert plan.stats(i) == stats_alone[i]
        assert any(len(a) > 0 for a in alone)


def test_graph_replay_follows_new_inputs(pkg, spectra):
    op = _params()
    p = jerk_params(op, sum(LENGTHS))
    p.max_batch = len(LENGTHS)
    # same lengths, different data: a new set of spectra with the same sizes
    other = [synth.spectrum(n, 900 + i, [synth.Signal(n / 5 + 0.5, 2.0, 0.0, 40.0, 1.0)])
             for i, n in enumerate(LENGTHS)]
    with pkg.Plan(p) as plan:
        alone_other, _ = _alone(pkg, plan, other)
        plan.search_batch([torch.from_numpy(F).cuda() for F in spectra], graph=True)
        plan.candidates()
        plan.search_batch([torch.from_numpy(F).cuda() for F in other], graph=True)   # replay
        cands = plan.candidates()
    for i in range(len(other)):
        assert [(0,) + _key(c)[1:] for c in cands if c.item == i] == alone_other[i]


def test_batch_item_matches_oracle(pkg, spectra):
    op = _params()
    p = jerk_params(op, sum(LENGTHS))
    p.max_batch = len(LENGTHS)
    i = 1
    res = oracle.search(spectra[i], op, keep_plane=True)
    tol = PLANE_TOL * res.plane.max()
    with pkg.Plan(p) as plan:
        plan.search_batch([torch.from_numpy(F).cuda() for F in spectra])
        cands = [c for c in plan.candidates() if c.item == i]
        for si, H in enumerate(op.stages):
            M, t = plan.maxproj(si, item=i)
            Mo, to = res.maxproj[H]
            assert np.max(np.abs(M.astype(np.float64) - Mo)) <= tol
    compare_candidates(cands, res, tol)


def test_batch_limits(pkg, spectra):
    from paper_1911_01353_gb300 import jerk
    op = _params()
    p = jerk_params(op, 40000)
    p.max_batch = 2
    with pkg.Plan(p) as plan:
        dev = [torch.from_numpy(F).cuda() for F in spectra[:4]]
        with pytest.raises(jerk.JerkError) as e:          # three spectra, max_batch 2
            plan.search_batch(dev[:3])
        assert e.value.code == jerk.JERK_EINVAL
        with pytest.raises(jerk.JerkError) as e:          # 30000 + 17777 > 40000 bins
            plan.search_batch(dev[:2])
        assert e.value.code == jerk.JERK_EINVAL
        plan.search_batch([dev[1], dev[3]])                # 17777 + 1025 fits
        assert {c.item for c in plan.candidates()} <= {0, 1}
