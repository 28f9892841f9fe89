"""Serving support through the C ABI: plans sharing one template bank,
per-spectrum sub-grids of the bank, transient launch tables, and the
continuous-batching server.

* a plan made by jerk_plan_share gives bitwise the parent's results, and the
  bank outlives whichever plan is destroyed first;
* a spectrum searched over a sub-grid |z| <= zs, |w| <= ws of a larger bank
  matches the FP64 oracle run with zmax = zs, wmax = ws (powers within
  PLANE_TOL of the plane maximum, candidates exact outside the guard band);
* every spectrum of a batch with mixed lengths and sub-grids gives bitwise
  what it gives searched alone, with cached, transient and graph tables;
* requests served by the server while others are on the GPU give bitwise
  what each gives alone.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import PLANE_TOL, compare_candidates, compare_maxproj, jerk_params, lib_ready

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BANK = dict(zmax=20, dz=2, wmax=60, dw=20)
LENGTHS = (30000, 17777, 50001, 1025, 8192, 24000)
SUBGRIDS = ((20, 60), (10, 20), (0, 0), (20, 0), (4, 40), (12, 60))


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib_ready()


@pytest.fixture(scope="module")
def spectra():
    out = []
    for i, n in enumerate(LENGTHS):
        sig = [synth.Signal(n / 3 + 0.25 * i, 4.0 - 2 * i, 20.0 * (i % 3 - 1), 30.0 + i, 0.3 * i),
               synth.Signal(n / 5 + 0.5, 0.0, 0.0, 25.0, 1.0)]
        out.append(synth.spectrum(n, 500 + i, sig, harmonics=2))
    return out


def bank_params(mode="abs", stages=(1, 2)):
    th = (12.0, 17.0) if mode == "abs" else (5.0, 5.0)
    return oracle.Params(BANK["zmax"], BANK["dz"], BANK["wmax"], BANK["dw"], stages=stages, thresh_mode=mode,
                         thresh=th[:len(stages)])


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def key(c):
    return (int(c.stage), int(c.p), int(c.t), float(c.power))


def to_sub(t, zs, ws):
    """Bank template index -> index in the sub-grid |z| <= zs, |w| <= ws."""
    nz = 2 * BANK["zmax"] // BANK["dz"] + 1
    z = -BANK["zmax"] + (t % nz) * BANK["dz"]
    w = -BANK["wmax"] + (t // nz) * BANK["dw"]
    i = (z + zs) // BANK["dz"]
    j = (w + ws) // BANK["dw"]
    return j * (2 * zs // BANK["dz"] + 1) + i


class _Rec:
    def __init__(self, c, t):
        self.stage, self.p, self.t, self.power = c.stage, c.p, t, c.power


def alone(plan, F, zs, ws):
    plan.search_batch([dev(F)], zmax=[zs], wmax=[ws])
    recs = plan.candidates()
    ns = int(plan.params.n_stages)
    mp = [tuple(a.copy() for a in plan.maxproj(si, 0)) for si in range(ns)]
    return [key(c) for c in recs], plan.stats(0), mp


def test_shared_plan_matches_parent(pkg, spectra):
    op = bank_params("sigma")
    p = jerk_params(op, 1 << 16)
    parent = pkg.Plan(p)
    p2 = jerk_params(op, 1 << 17)
    p2.max_batch = 4
    child = parent.share(p2)
    assert child.info.d_bank == parent.info.d_bank and child.info.bank_bytes == parent.info.bank_bytes
    F = spectra[2]
    parent.search(dev(F))
    want = [key(c) for c in parent.candidates()]
    want_stats = parent.stats(0)
    want_M = [parent.maxproj(si)[0].copy() for si in range(2)]
    parent.close()                                   # the bank stays with the child
    child.search(dev(F))
    assert [key(c) for c in child.candidates()] == want
    assert child.stats(0) == want_stats
    for si in range(2):
        assert np.array_equal(child.maxproj(si)[0], want_M[si])
    child.close()
    assert len(want) > 0


def test_share_rejects_other_bank(pkg):
    from paper_1911_01353_gb300 import jerk
    op = bank_params()
    with pkg.Plan(jerk_params(op, 1 << 14)) as parent:
        for field, value in (("zmax", 10), ("wmax", 40), ("dz", 4), ("n_stages", 1), ("seg_len", 1024)):
            q = jerk_params(op, 1 << 14)
            setattr(q, field, value)
            with pytest.raises(jerk.JerkError) as e:
                parent.share(q)
            assert e.value.code == jerk.JERK_EINVAL


@pytest.mark.parametrize("zs,ws", [(10, 20), (0, 0), (20, 0), (4, 40)])
def test_subgrid_matches_oracle(pkg, spectra, zs, ws):
    op = bank_params()
    F = spectra[0]
    sub = oracle.Params(zs, BANK["dz"], ws, BANK["dw"], stages=op.stages, thresh_mode=op.thresh_mode,
                        thresh=op.thresh)
    res = oracle.search(F, sub, keep_plane=True)
    tol = PLANE_TOL * res.plane.max()
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        plan.search_batch([dev(F)], zmax=[zs], wmax=[ws])
        recs = plan.candidates()
        for si, H in enumerate(op.stages):
            M, t = plan.maxproj(si)
            Mo, to = res.maxproj[H]
            fund, S = res.sums[H]
            compare_maxproj(M, to_sub(t.astype(np.int64), zs, ws), Mo, to, S, tol)
    for c in recs:                                   # every candidate lies inside the sub-grid
        assert abs(c.z) <= zs and abs(c.w) <= ws
    compare_candidates([_Rec(c, to_sub(c.t, zs, ws)) for c in recs], res, tol)
    assert len(res.candidates) > 0


@pytest.mark.parametrize("mode", ["abs", "sigma"])
def test_subgrid_mix_equals_alone(pkg, spectra, mode):
    op = bank_params(mode)
    p = jerk_params(op, sum(LENGTHS))
    p.max_batch = len(LENGTHS)
    zm = [zw[0] for zw in SUBGRIDS]
    wm = [zw[1] for zw in SUBGRIDS]
    with pkg.Plan(p) as plan:
        ref = [alone(plan, F, zs, ws) for F, zs, ws in zip(spectra, zm, wm)]
        dv = [dev(F) for F in spectra]
        for flags in (dict(), dict(transient=True), dict(graph=True), dict(graph=True), dict(transient=True)):
            plan.search_batch(dv, zmax=zm, wmax=wm, **flags)
            recs = plan.candidates()
            for i in range(len(spectra)):
                assert [key(c) for c in recs if c.item == i] == ref[i][0], (flags, i)
                assert plan.stats(i) == ref[i][1], (flags, i)
                for si in range(len(op.stages)):
                    M, t = plan.maxproj(si, item=i)
                    assert np.array_equal(M, ref[i][2][si][0]) and np.array_equal(t, ref[i][2][si][1])
    assert sum(len(r[0]) for r in ref) > 0


def test_whole_bank_subgrid_is_the_plain_search(pkg, spectra):
    op = bank_params()
    F = spectra[1]
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        plan.search(dev(F))
        want = [key(c) for c in plan.candidates()]
        plan.search_batch([dev(F)], zmax=[BANK["zmax"]], wmax=[BANK["wmax"]], transient=True)
        assert [key(c) for c in plan.candidates()] == want


def test_subgrid_argument_errors(pkg, spectra):
    from paper_1911_01353_gb300 import jerk
    op = bank_params()
    p = jerk_params(op, 1 << 17)
    p.max_batch = 2
    with pkg.Plan(p) as plan:
        x = dev(spectra[0])
        for zs, ws in ((3, 0), (22, 0), (0, 30), (0, 80), (-2, 0)):
            with pytest.raises(jerk.JerkError) as e:
                plan.search_batch([x], zmax=[zs], wmax=[ws])
            assert e.value.code == jerk.JERK_EINVAL
        with pytest.raises(jerk.JerkError) as e:
            plan.search_batch([x], zmax=[10], wmax=[20], graph=True, transient=True)
        assert e.value.code == jerk.JERK_EINVAL


def test_server_mix_equals_alone(pkg, spectra):
    from paper_1911_01353_gb300 import jerk, serve
    rng = np.random.default_rng(7)
    srv = serve.Server(BANK["zmax"], BANK["wmax"], dz=BANK["dz"], dw=BANK["dw"], stages=(1, 2),
                       thresh=(12.0, 17.0), thresh_mode=jerk.THRESH_ABS, n_workers=3, worker_bins=1 << 17, max_batch=4,
                       max_candidates=1 << 16, reserve_bytes=1 << 28, small_cells=2e6)
    try:
        reqs = []
        for k in range(18):
            F = spectra[k % len(spectra)]
            zs, ws = SUBGRIDS[rng.integers(len(SUBGRIDS))]
            reqs.append(serve.Request(k, F, zs, ws, arrival=float(rng.uniform(0.0, 0.2))))
        done = srv.run(reqs)
        assert sorted(r.rid for r in done) == list(range(18))
        for r in done:
            want, want_stats = srv.alone(r)
            assert r.candidates == [(s, p, t, pw) for (s, p, t, pw) in want], r.rid
            assert r.stats == want_stats, r.rid
            assert r.done >= r.dispatched >= r.admitted >= r.arrival
        st = serve.summary(done, BANK["dz"], BANK["dw"])
        assert st["cells"] == sum(serve.cells_of(r, BANK["dz"], BANK["dw"]) for r in done)
        assert st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        srv.close()
