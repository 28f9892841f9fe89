"""Parity at the benchmark's full size, in the configuration bench.py times:
a 2^22-bin spectrum with 8 injected chirps, zmax 200 / wmax 600 (12 261
templates, L = 4096), stages 1-2-4-8, SIGMA thresholds T = 19, 17, 15, 14.

The oracle cannot compute the 411 GB plane, so it checks sampled outputs one
by one (direct correlation in FP64) and properties that hold at any size:

* plane rows of boundary and random templates (jerk_plane, the search's own
  kernel in plane-write mode) at thousands of sampled cells;
* the max-projections of every stage at sampled cells: the value equals the
  oracle's power (or harmonic sum) of the reported argmax, and bounds the
  oracle's value at many other templates (fundamentals);
* every stage-1 candidate's power equals the oracle's at its (p, t), and the
  candidates satisfy the peak rule on the GPU's own max-projection;
* the injected signals show in the max-projection at their frequencies;
* the statistics are those of unit noise (mean = tap energy, sigma = mean)
  and grow as H and sqrt(H) over the stages;
* against the oracle's whole-bank result by its FFT route (stored under
  tests/golden/ by make_paper_scale.py): the candidate list of every stage
  exactly (outside a guard band around FP32 decisions), mu_H and sigma_H, and
  M_H with its argmax at 2^16 sampled cells per stage.

Tolerance: PLANE_TOL of the plane maximum per power, H times that for a sum
of H powers; the reduced-precision filters with their own bounds.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from parity import PLANE_TOL, jerk_params, lib_ready

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

T_SIGMA = (19.0, 17.0, 15.0, 14.0)
TC_TOL = {1: 1e-2, 2: 1e-3}


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib_ready()


@pytest.fixture(scope="module")
def full(pkg):
    wl = synth.paper_scale()
    F = wl.make()
    op = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=wl.stages, thresh_mode="sigma", thresh=T_SIGMA)
    Fn = oracle.normalise(F, op.norm_block)
    x = torch.from_numpy(F).cuda()
    plan = pkg.Plan(jerk_params(op, F.size, max_candidates=1 << 20))
    plan.search(x)
    cands = plan.candidates()
    M = [plan.maxproj(si) for si in range(len(op.stages))]          # (value, argmax t) per stage
    stats = plan.stats(0)
    yield dict(wl=wl, F=F, Fn=Fn, op=op, x=x, plan=plan, cands=cands, M=M, stats=stats)
    plan.close()


def test_full_size_plane_rows(full):
    op, Fn, plan, x = full["op"], full["Fn"], full["plan"], full["x"]
    T, bN = op.n_templates, 2 * full["F"].size
    rng = np.random.default_rng(21)
    picks = [0, T - 1, op.nz - 1, T - op.nz, T // 2] + [int(t) for t in rng.choice(T, 3, replace=False)]
    bank = oracle.Bank(op, templates=picks)
    scale = float(full["M"][0][0].max())                              # the plane maximum
    tol = PLANE_TOL * scale
    sig = [int(2 * s.r) for s in full["wl"].signals]
    out = torch.empty(bN, dtype=torch.float32, device="cuda")
    for t in picks:
        plan.plane(x, t, 1, out)
        row = out.cpu().numpy()
        ps = np.concatenate([rng.integers(0, bN, 3000), [0, 1, bN - 2, bN - 1],
                             np.concatenate([np.arange(p - 8, p + 9) for p in sig])])
        want = bank.power_cells(Fn, np.full(ps.size, t), ps)
        err = np.abs(row[ps].astype(np.float64) - want)
        assert err.max() <= tol, (t, float(err.max()), tol)


def test_full_size_maxproj_samples(full):
    op, Fn, M = full["op"], full["Fn"], full["M"]
    rng = np.random.default_rng(22)
    bN = 2 * full["F"].size
    tol = PLANE_TOL * float(M[0][0].max())
    cand_p = [int(c.p) for c in full["cands"] if c.stage == 1][:40]
    cells = np.concatenate([rng.integers(0, bN, 60), cand_p]).astype(np.int64)
    # stage 1: the argmax's power equals M1; random templates never exceed it
    R = [int(t) for t in rng.choice(op.n_templates, 600, replace=False)]
    arg = [int(M[0][1][p]) for p in cells]
    bank = oracle.Bank(op, templates=sorted(set(R) | set(arg)))
    got = M[0][0][cells].astype(np.float64)
    at_arg = bank.power_cells(Fn, arg, cells)
    assert np.max(np.abs(at_arg - got)) <= tol
    tt = np.repeat(np.array(R), cells.size)
    pp = np.tile(cells, len(R))
    others = bank.power_cells(Fn, tt, pp).reshape(len(R), cells.size)
    assert np.all(others <= got[None, :] + tol)
    # stages H > 1: S_H(p, f) = sum_h P(h p, t(h z_f, h w_f))
    for si, H in enumerate(op.stages):
        if H == 1:
            continue
        fund, harm = oracle.stage_templates(op, H)
        ncell = (bN - 1) // H + 1
        cs = np.concatenate([rng.integers(0, ncell, 40), rng.integers(max(0, ncell - 50), ncell, 4)])
        row_of = {int(f): i for i, f in enumerate(fund)}
        fr = [int(f) for f in rng.choice(fund, min(150, fund.size), replace=False)]
        argf = [int(M[si][1][p]) for p in cs]
        need = sorted({int(t) for f in set(fr) | set(argf) for t in harm[row_of[f]]})
        bk = oracle.Bank(op, templates=need)

        def S(fs, ps):
            tot = np.zeros(len(fs))
            for h in range(1, H + 1):
                tot += bk.power_cells(Fn, [harm[row_of[f]][h - 1] for f in fs], [h * p for p in ps])
            return tot

        gotH = M[si][0][cs].astype(np.float64)
        assert np.max(np.abs(S(argf, cs) - gotH)) <= H * tol, H
        fs = np.repeat(np.array(fr), cs.size)
        ps = np.tile(cs, len(fr))
        assert np.all(S(list(fs), list(ps)).reshape(len(fr), cs.size) <= gotH[None, :] + H * tol), H


def test_full_size_candidates(full):
    op, Fn, M, cands = full["op"], full["Fn"], full["M"], full["cands"]
    tol = PLANE_TOL * float(M[0][0].max())
    mu, sd, theta = full["stats"]
    c1 = [c for c in cands if c.stage == 1]
    assert c1
    bank = oracle.Bank(op, templates=sorted({int(c.t) for c in c1}))
    want = bank.power_cells(Fn, [int(c.t) for c in c1], [int(c.p) for c in c1])
    assert np.max(np.abs(want - np.array([c.power for c in c1]))) <= tol
    for si, H in enumerate(op.stages):
        Mv = M[si][0]
        for c in (c for c in cands if c.stage == H):
            p = int(c.p)
            assert Mv[p] > theta[si] and Mv[p] == np.float32(c.power)
            assert p == 0 or Mv[p] > Mv[p - 1]
            assert p + 1 == Mv.size or Mv[p] >= Mv[p + 1]
    # the injected signals stand out in the stage-1 max-projection at their frequencies,
    # and those clearly above the threshold are candidates
    for s in full["wl"].signals:
        lo, hi = int(2 * s.r) - 4, int(2 * s.r) + 5
        peak = float(M[0][0][lo:hi].max())
        assert peak >= 0.5 * s.snr, (s.r, s.snr, peak)
        if peak > theta[0] + 2 * tol:
            assert any(lo <= c.p < hi for c in c1), (s.r, peak)


def test_full_size_statistics(full):
    mu, sd, theta = full["stats"]
    op = full["op"]
    assert 0.98 < mu[0] < 1.01 and 0.97 < sd[0] / mu[0] < 1.05           # Exp-like unit noise
    for si, H in enumerate(op.stages):
        assert mu[si] == pytest.approx(H * mu[0], rel=0.03)
        assert sd[si] == pytest.approx(math.sqrt(H) * sd[0], rel=0.05)
        assert theta[si] == pytest.approx(mu[si] + T_SIGMA[si] * sd[si], rel=1e-5)


def _golden():
    """The FP64 oracle's result for this workload by its FFT route, written by
    tests/golden/make_paper_scale.py (which calls only oracle/ and synth/)."""
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    with open(os.path.join(here, "paper_scale_candidates.json")) as f:
        g = json.load(f)
    return g, np.load(os.path.join(here, "paper_scale_maxproj_sample.npz"))


def test_golden_matches_this_workload(full):
    g, _ = _golden()
    q, op = g["params"], full["op"]
    assert g["workload"] == full["wl"].name
    assert (q["zmax"], q["dz"], q["wmax"], q["dw"], tuple(q["stages"]), q["thresh_mode"], tuple(q["thresh"]),
            q["norm_block"], q["pad_bins"]) == (op.zmax, op.dz, op.wmax, op.dw, tuple(op.stages), op.thresh_mode,
                                                tuple(op.thresh), op.norm_block, op.pad_bins)


def test_full_size_statistics_equal_oracle(full):
    """mu_H and sigma_H of every stage against the oracle's FP64 values over
    all 1.03e11 stage-1 cells (and every defined cell of S_2, S_4, S_8)."""
    g, _ = _golden()
    mu, sd, theta = full["stats"]
    for si, H in enumerate(full["op"].stages):
        st = g["stages"][str(H)]
        assert mu[si] == pytest.approx(st["mu"], rel=1e-5), H
        assert sd[si] == pytest.approx(st["sigma"], rel=1e-5), H
        assert theta[si] == pytest.approx(st["theta"], rel=1e-5), H


def test_full_size_candidates_equal_oracle_list(full):
    """The GPU's candidate list against the oracle's, exactly: every oracle
    candidate is found with the same template and its power within H x the
    tolerance, and every GPU candidate is an oracle candidate.  A cell is
    guarded (left out) only when one of its decisions -- above theta, above
    the left neighbour, not below the right one -- is within 2 H x the
    tolerance of flipping in the oracle (theta widened by the GPU's own
    difference from the oracle's theta); the template is compared wherever the
    oracle's best and runner-up differ by more than that."""
    g, _ = _golden()
    tol = PLANE_TOL * g["plane_max"]
    mu, sd, theta = full["stats"]
    got = {(int(c.stage), int(c.p)): (int(c.t), float(c.power)) for c in full["cands"]}
    total = guarded = 0
    for si, H in enumerate(full["op"].stages):
        st = g["stages"][str(H)]
        band = 2 * H * tol
        dth = abs(float(theta[si]) - st["theta"])
        want = {r[0]: r for r in st["candidates"]}
        near = {r[0]: r for r in st["near"]}

        def is_guarded(r):
            p, t, m, sec, left, right = r
            left = -np.inf if left is None else left
            right = -np.inf if right is None else right
            return abs(m - st["theta"]) <= band + dth or abs(m - left) <= band or abs(m - right) <= band

        for p, r in want.items():
            total += 1
            if is_guarded(r):
                guarded += 1
                continue
            assert (H, p) in got, "oracle candidate (H=%d, p=%d, M=%g) missing on the GPU" % (H, p, r[2])
            t, power = got[(H, p)]
            assert abs(power - r[2]) <= H * tol, (H, p, power, r[2])
            if r[2] - r[3] > band:
                assert t == r[1], "template differs at (H=%d, p=%d): %d vs %d" % (H, p, t, r[1])
        for (h, p) in got:
            if h != H or p in want:
                continue
            assert p in near and is_guarded(near[p]), "GPU candidate (H=%d, p=%d) is not an oracle candidate" % (H, p)
            guarded += 1
    assert total > 100
    assert guarded <= max(4, total // 50), (guarded, total)


def test_full_size_maxproj_equals_oracle_sample(full):
    """M_H and its argmax at the stored cells (65 536 random cells per stage
    plus +-4 around every candidate) against the oracle's FFT-route values."""
    g, z = _golden()
    tol = PLANE_TOL * g["plane_max"]
    for si, H in enumerate(full["op"].stages):
        ps = z["p%d" % H].astype(np.int64)
        m, t, sec = z["m%d" % H].astype(np.float64), z["t%d" % H], z["s%d" % H].astype(np.float64)
        Mv, Mt = full["M"][si]
        assert Mv.size == g["stages"][str(H)]["cells"]
        err = np.abs(Mv[ps].astype(np.float64) - m)
        assert err.max() <= H * tol, (H, float(err.max()))
        sure = m - sec > 2 * H * tol
        assert sure.mean() > 0.5
        bad = np.nonzero(sure & (Mt[ps] != t))[0]
        assert bad.size == 0, (H, ps[bad[:5]], Mt[ps][bad[:5]], t[bad[:5]])


@pytest.mark.parametrize("prec", [1, 2])
def test_full_size_tensor_core_rows(full, pkg, prec):
    op, Fn, x = full["op"], full["Fn"], full["x"]
    T, bN = op.n_templates, 2 * full["F"].size
    # plane rows do not depend on the stages: a stage-1 plan needs no harmonic-row workspace
    op1 = oracle.Params(op.zmax, op.dz, op.wmax, op.dw, stages=(1,), thresh=(20.0,))
    p = jerk_params(op1, full["F"].size)
    p.precision = prec
    rng = np.random.default_rng(23)
    picks = [0, T // 2, int(rng.integers(T))]
    bank = oracle.Bank(op, templates=picks)
    scale = float(full["M"][0][0].max())
    out = torch.empty(bN, dtype=torch.float32, device="cuda")
    with pkg.Plan(p) as plan:
        for t in picks:
            plan.plane(x, t, 1, out)
            ps = rng.integers(0, bN, 3000)
            want = bank.power_cells(Fn, np.full(ps.size, t), ps)
            err = np.abs(out.cpu().numpy()[ps].astype(np.float64) - want)
            assert err.max() <= TC_TOL[prec] * scale, (prec, t, float(err.max()) / scale)


def test_dm_batch_configuration(pkg):
    """The batched configuration (zmax 200, wmax 300: 6 231 templates, stages
    1-2-4-8, SIGMA), three DM-trial spectra of 2^20 - 2^21 bins in one graph-
    replayed launch: each item's candidates are exactly its own search's, and
    the oracle agrees with sampled max-projection cells and every stage-1
    candidate's power."""
    trials = synth.dm_trials(3, seed=3, lo=20.0, hi=21.0)
    specs = [synth.spectrum(n, seed, sigs) for n, seed, sigs in trials]
    op = oracle.Params(200, 2, 300, 20, stages=(1, 2, 4, 8), thresh_mode="sigma", thresh=T_SIGMA)
    p = jerk_params(op, sum(s.size for s in specs), max_candidates=1 << 20)
    p.max_batch = len(specs)
    rng = np.random.default_rng(24)
    with pkg.Plan(p) as plan:
        dev = [torch.from_numpy(s).cuda() for s in specs]
        alone = []
        for x in dev:
            plan.search(x)
            alone.append([(c.stage, c.p, c.t, c.power) for c in plan.candidates()])
        plan.search_batch(dev, graph=True)
        plan.search_batch(dev, graph=True)                             # the replay
        recs = plan.candidates()
        Ms = [plan.maxproj(0, item=i) for i in range(len(specs))]
    for i, F in enumerate(specs):
        mine = [(c.stage, c.p, c.t, c.power) for c in recs if c.item == i]
        assert mine == alone[i], i
        Fn = oracle.normalise(F, op.norm_block)
        M, t = Ms[i]
        tol = PLANE_TOL * float(M.max())
        cells = rng.integers(0, M.size, 80)
        c1 = [c for c in recs if c.item == i and c.stage == 1]
        bank = oracle.Bank(op, templates=sorted({int(t[p]) for p in cells} | {int(c.t) for c in c1}))
        assert np.max(np.abs(bank.power_cells(Fn, t[cells], cells) - M[cells])) <= tol
        if c1:
            want = bank.power_cells(Fn, [int(c.t) for c in c1], [int(c.p) for c in c1])
            assert np.max(np.abs(want - np.array([c.power for c in c1]))) <= tol


def test_served_size_subgrid_request(pkg):
    """A serving-size request: the (300, 900) bank (27 391 templates) searches
    a 2^22-bin spectrum over its (200, 600) sub-grid at stage 1, as the server
    does; sampled cells and every candidate agree with the oracle's direct
    correlation, and every reported template lies inside the sub-grid."""
    wl = synth.paper_scale()
    F = wl.make()
    op = oracle.Params(300, 2, 900, 20, stages=(1,), thresh_mode="sigma", thresh=(19.0,))
    with pkg.Plan(jerk_params(op, F.size, max_candidates=1 << 20)) as plan:
        plan.search_batch([torch.from_numpy(F).cuda()], zmax=[200], wmax=[600], transient=True)
        recs = plan.candidates()
        M, t = plan.maxproj(0)
    Fn = oracle.normalise(F, op.norm_block)
    tol = PLANE_TOL * float(M.max())
    rng = np.random.default_rng(25)
    cells = rng.integers(0, M.size, 80)
    zt, wt = oracle.grid(op)
    assert all(abs(zt[t[p]]) <= 200 and abs(wt[t[p]]) <= 600 for p in cells)
    assert recs and all(abs(c.z) <= 200 and abs(c.w) <= 600 for c in recs)
    bank = oracle.Bank(op, templates=sorted({int(t[p]) for p in cells} | {int(c.t) for c in recs}))
    assert np.max(np.abs(bank.power_cells(Fn, t[cells], cells) - M[cells])) <= tol
    want = bank.power_cells(Fn, [int(c.t) for c in recs], [int(c.p) for c in recs])
    assert np.max(np.abs(want - np.array([c.power for c in recs]))) <= tol


def test_full_size_split_by_template_range(full):
    """The benchmark's search split in two template ranges (as two GPUs would
    run it), merged: max-projections bitwise equal to the whole-bank search,
    statistics to the order of FP64 additions, the same candidates.  Runs on
    the fixture's plan, so it comes last in this file."""
    from test_gpu_split import compare, split_search

    from paper_1911_01353_gb300.ranks import template_range
    plan, x = full["plan"], full["x"]
    T = plan.info.n_templates
    split_search(plan, x, [template_range(T, r, 2) for r in range(2)])
    compare(plan, full["M"], full["cands"], full["stats"], True)
