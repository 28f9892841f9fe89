"""Reduced-precision filter (BF16 / FP16 tensor-core DFT blocks, FP32
accumulation) vs the FP64 oracle, through the C ABI.

The tensor-core path rounds the template products and the intermediate
spectra to 16 bits, so its powers carry that rounding: with 8 (BF16) or 11
(FP16) significant bits an element is off by up to 2^-9 or 2^-12 relative,
and two 64-point blocks accumulate that over ~sqrt(2 * 64) terms.  The
bounds below, relative to the plane maximum, are 4-5x the largest errors
measured on the 2^16-bin workload (BF16 2.3e-3, FP16 1.9e-4).  Candidates
are compared exactly outside the same guard band as the FP32 path, with the
tolerance of the precision.  Everything else -- grouping, batching,
sub-grids, statistics -- is shared with the FP32 path and must behave the
same way (a batch gives bitwise the results of its items alone).
"""
import numpy as np
import pytest

import oracle
import synth
from parity import compare_candidates, compare_maxproj, jerk_params, lib_ready, oracle_params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {1: 1e-2, 2: 1e-3}           # max |P - P_oracle| / max P_oracle
STAT_TOL = {1: 5e-3, 2: 5e-4}      # relative, mean and standard deviation (BF16 rounding biases powers up)
NAME = {1: "bf16", 2: "fp16"}


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib_ready()


@pytest.fixture(scope="module")
def small():
    wl = synth.small_single()
    F = wl.make()
    op = oracle_params(wl)
    return F, op, oracle.search(F, op, keep_plane=True)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def tc_params(op, n, prec, **kw):
    p = jerk_params(op, n, **kw)
    p.precision = prec
    return p


@pytest.mark.parametrize("prec", [1, 2], ids=lambda p: NAME[p])
def test_plane_error_bound(pkg, small, prec):
    F, op, res = small
    with pkg.Plan(tc_params(op, F.size, prec)) as plan:
        assert plan.info.seg_len == 4096
        T = plan.info.n_templates
        out = torch.empty((T, 2 * F.size), dtype=torch.float32, device="cuda")
        plan.plane(dev(F), 0, T, out)
        P = out.cpu().numpy().astype(np.float64)
    pmax = res.plane.max()
    err = np.abs(P - res.plane)
    assert err.max() <= TOL[prec] * pmax, "%s max error %.3g of the plane max" % (NAME[prec], err.max() / pmax)
    # the error is rounding noise, not a bias: RMS well below the bound
    assert np.sqrt((err ** 2).mean()) <= 0.1 * TOL[prec] * pmax


@pytest.mark.parametrize("prec", [1, 2], ids=lambda p: NAME[p])
def test_maxproj_and_candidates(pkg, small, prec):
    F, op, res = small
    tol = TOL[prec] * res.plane.max()
    with pkg.Plan(tc_params(op, F.size, prec)) as plan:
        plan.search(dev(F))
        cands = plan.candidates()
        for si, H in enumerate(op.stages):
            M, t = plan.maxproj(si)
            Mo, to = res.maxproj[H]
            fund, S = res.sums[H]
            compare_maxproj(M, t, Mo, to, S, tol)
    compare_candidates(cands, res, tol)
    # the injected signal is found, at its template or (BF16: the neighbouring
    # templates' powers are within the rounding of the peak's) one grid step away
    assert any(c.stage == 1 and abs(c.r - 10000.25) < 1.0 and abs(c.z - 12) <= 2 and abs(c.w - 40) <= 20
               for c in cands)


@pytest.mark.parametrize("prec", [1, 2], ids=lambda p: NAME[p])
def test_ragged_sigma_statistics(pkg, prec):
    n = 50001                                       # many segments, ragged tail
    F = synth.spectrum(n, 77, [synth.Signal(20000.5, -6.0, 20.0, 40.0, 0.4)], harmonics=2)
    op = oracle.Params(12, 2, 40, 20, stages=(1, 2), thresh_mode="sigma", thresh=(6.0, 6.0))
    res = oracle.search(F, op, keep_plane=True)
    tol = TOL[prec] * res.plane.max()
    with pkg.Plan(tc_params(op, n, prec)) as plan:
        plan.search(dev(F))
        cands = plan.candidates()
        mu, sd, th = plan.stats(0)
    for si, H in enumerate(op.stages):
        mo, so = res.stats[H]
        # statistics are means over millions of cells: far tighter than one cell, but
        # the power rounding error adds E|e|^2 > 0 to every cell (a bias, not noise)
        assert abs(mu[si] - mo) <= STAT_TOL[prec] * mo
        assert abs(sd[si] - so) <= STAT_TOL[prec] * so
    compare_candidates(cands, res, tol)


@pytest.mark.parametrize("prec", [1, 2], ids=lambda p: NAME[p])
def test_batch_and_subgrids_equal_alone(pkg, prec):
    lengths = (30000, 8192, 17777)
    specs = [synth.spectrum(n, 900 + i, [synth.Signal(n / 3 + 0.5, 2.0 * i, 20.0, 35.0, 0.1)])
             for i, n in enumerate(lengths)]
    op = oracle.Params(20, 2, 60, 20, stages=(1, 2), thresh=(12.0, 17.0))
    p = tc_params(op, sum(lengths), prec)
    p.max_batch = len(lengths)
    zm, wm = [20, 10, 4], [60, 20, 0]

    def key(c):
        return (int(c.stage), int(c.p), int(c.t), float(c.power))

    with pkg.Plan(p) as plan:
        alone = []
        for F, zs, ws in zip(specs, zm, wm):
            plan.search_batch([dev(F)], zmax=[zs], wmax=[ws])
            alone.append(([key(c) for c in plan.candidates()], plan.stats(0)))
        for flags in (dict(), dict(transient=True), dict(graph=True)):
            plan.search_batch([dev(F) for F in specs], zmax=zm, wmax=wm, **flags)
            recs = plan.candidates()
            for i in range(len(specs)):
                assert [key(c) for c in recs if c.item == i] == alone[i][0], (flags, i)
                assert plan.stats(i) == alone[i][1]
    assert sum(len(a[0]) for a in alone) > 0


def test_precision_argument_checks(pkg):
    from paper_1911_01353_gb300 import jerk
    op = oracle.Params(4, 2, 0, 20, stages=(1,), thresh=(10.0,))
    for prec, seg in ((3, 0), (-1, 0), (1, 2048), (2, 8192)):
        with pytest.raises(jerk.JerkError) as e:
            pkg.Plan(tc_params(op, 4096, prec, seg_len=seg))
        assert e.value.code == jerk.JERK_EINVAL
    with pkg.Plan(tc_params(op, 4096, 2, seg_len=4096)) as plan:
        assert plan.info.seg_len == 4096
