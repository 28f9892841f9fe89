"""Power at arbitrary (r, z, w) points, off-grid refinement and the 3-D
26-neighbour peak test, through the C ABI, against the FP64 oracle.

* on the grid the direct evaluation is the plane: equal to the oracle's plane
  and to the fused filter's plane within PLANE_TOL of the plane maximum;
* off the grid it equals the oracle's direct evaluation within the same
  bound (FP32 products, FP64 sums, quadrature of the template bank);
* refining the candidate of the 2^16-bin workload lands nearer the injected
  signal's r = 10000.25 (a quarter bin, between two cells) than the cell
  spacing, and agrees with the oracle's refinement on the same grid;
* the 26-neighbour test agrees with the oracle's wherever the decision is
  not within the tolerance of a tie.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import PLANE_TOL, jerk_params, lib_ready, oracle_params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
    res = oracle.search(F, op, keep_plane=True)
    return wl, F, op, res, oracle.normalise(F, op.norm_block)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_power_at_on_grid_is_the_plane(pkg, small):
    wl, F, op, res, Fn = small
    zt, wt = oracle.grid(op)
    rng = np.random.default_rng(3)
    T, bN = res.plane.shape
    ts = rng.integers(0, T, 150)
    ps = rng.integers(0, bN, 150)
    ps[:20] = rng.integers(19990, 20010, 20)                 # around the signal
    ps[20:25] = [0, 1, bN - 1, bN - 2, 3]                    # spectrum edges
    pts = np.stack([ps / 2.0, zt[ts], wt[ts]], axis=1).astype(np.float64)
    tol = PLANE_TOL * res.plane.max()
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        x = dev(F)
        got = plan.power_at(x, pts).astype(np.float64)
        out = torch.empty((T, bN), dtype=torch.float32, device="cuda")
        plan.plane(x, 0, T, out)
        gpu_plane = out.cpu().numpy()
    want = res.plane[ts, ps]
    assert np.max(np.abs(got - want)) <= tol
    assert np.max(np.abs(got - gpu_plane[ts, ps])) <= tol


def test_power_at_off_grid_matches_oracle(pkg, small):
    wl, F, op, res, Fn = small
    rng = np.random.default_rng(4)
    pts = np.stack([rng.uniform(9990, 10010, 40), rng.uniform(-20, 20, 40), rng.uniform(-60, 60, 40)], axis=1)
    pts = np.concatenate([pts, [[10000.25, 12.0, 40.0], [10000.3, 11.7, 37.5], [3.1, 0.5, -7.0],
                                [65534.6, -3.3, 1.0], [500.123, 19.9, -59.9]]])
    want = np.array([oracle.power_at(Fn, *p, pad=op.pad_bins) for p in pts])
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        got = plan.power_at(dev(F), pts).astype(np.float64)
    assert np.max(np.abs(got - want)) <= PLANE_TOL * max(want.max(), res.plane.max())
    assert np.argmax(got) == np.argmax(want)


def test_refine_recovers_the_injected_signal(pkg, small):
    wl, F, op, res, Fn = small
    step, half = (0.05, 0.5, 5.0), (10, 3, 3)
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        x = dev(F)
        plan.search(x)
        cands = [c for c in plan.candidates() if c.stage == 1 and abs(c.r - 10000.25) < 2]
        assert cands
        c = max(cands, key=lambda c: c.power)
        ref = plan.refine(x, [c], step, half)[0]
    # noise (power SNR 30) moves the maximum by a fraction of a bin: closer than the cell spacing
    assert abs(ref.r - 10000.25) < 0.25 and abs(ref.z - 12) <= 1.5 and abs(ref.w - 40) <= 10.0
    assert ref.power >= ref.power_in and ref.power_in == pytest.approx(c.power, rel=1e-4)
    (r, z, w, P), centre = oracle.refine(Fn, c.r, float(c.z), float(c.w), step, half, pad=op.pad_bins)
    tol = PLANE_TOL * res.plane.max()
    assert abs(ref.power - P) <= tol and abs(ref.power_in - centre) <= tol
    # the same grid point, unless another is within the tolerance of the maximum
    same = abs(ref.r - r) < 1e-9 and abs(ref.z - z) < 1e-4 and abs(ref.w - w) < 1e-4
    assert same or abs(oracle.power_at(Fn, ref.r, ref.z, ref.w, pad=op.pad_bins) - P) <= 2 * tol


def test_26_neighbour_peaks(pkg, small):
    wl, F, op, res, Fn = small
    tol = PLANE_TOL * res.plane.max()
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        x = dev(F)
        plan.search(x)
        cands = [c for c in plan.candidates() if c.stage == 1][:12]
        refs = plan.refine(x, cands, (0.5, float(op.dz), float(op.dw)), (1, 1, 1))
    assert cands
    decided = 0
    for c, ref in zip(cands, refs):
        (r, z, w, P), centre = oracle.refine(Fn, c.r, float(c.z), float(c.w), (0.5, op.dz, op.dw), (1, 1, 1),
                                             pad=op.pad_bins)
        if abs(P - centre) <= 2 * tol and P != centre:
            continue                                           # a near tie: either answer is right
        decided += 1
        assert bool(ref.is_peak) == (centre >= P)
    assert decided > 0
    # the injected signal's cell is a 3-D peak
    best = max(zip(cands, refs), key=lambda cr: cr[0].power)
    assert best[1].is_peak == 1 or abs(best[0].r - 10000.25) > 1


def test_refine_argument_checks(pkg, small):
    from paper_1911_01353_gb300 import jerk
    wl, F, op, res, Fn = small
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        x = dev(F)
        plan.search(x)
        c = plan.candidates()[:1]
        for step, half in (((0.1, 1, 1), (65, 0, 0)), ((-0.1, 1, 1), (1, 1, 1)), ((float("nan"), 1, 1), (1, 1, 1))):
            with pytest.raises(jerk.JerkError) as e:
                plan.refine(x, c, step, half)
            assert e.value.code == jerk.JERK_EINVAL
        with pytest.raises(jerk.JerkError) as e:
            plan.power_at(x, [[100.0, 1e5, 0.0]])
        assert e.value.code == jerk.JERK_EINVAL
        assert plan.refine(x, [], (0.1, 1, 1), (1, 1, 1)) == []
