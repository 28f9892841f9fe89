"""One spectrum searched in parts by template range (jerk_search_range on each
range, an element-wise maximum of the packed max-projections and a sum of the
statistics, then jerk_select), as ranks on several GPUs would; here the parts
run one after another on one GPU, through the C ABI.  The merged
max-projections equal the whole-bank search's bitwise, and the candidates are
the same (outside the thresholds' last-bit difference from the order of FP64
additions)."""
import numpy as np
import pytest

import synth
from parity import jerk_params, lib_ready, oracle_params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib_ready()


def split_search(plan, x, ranges):
    """Partial searches over `ranges` on one plan, merged as the ranks would
    merge them; returns the merged sums."""
    ns = int(plan.params.n_stages)
    merged = None
    tot = np.zeros((3, ns))
    for lo, hi in ranges:
        plan.search_range(x, lo, hi)
        s1, s2, n = plan.range_sums()
        tot += np.stack([s1, s2, n])
        parts = [plan.maxproj_tensor(si).clone() for si in range(ns)]
        merged = parts if merged is None else [torch.maximum(a, b) for a, b in zip(merged, parts)]
    for si in range(ns):
        plan.maxproj_tensor(si).copy_(merged[si])
    torch.cuda.synchronize()
    plan.select(tot[0], tot[1], tot[2])
    return tot


def compare(plan, whole_M, whole_cands, whole_stats, sigma):
    ns = int(plan.params.n_stages)
    for si in range(ns):
        M, t = plan.maxproj(si)
        assert np.array_equal(M, whole_M[si][0]) and np.array_equal(t, whole_M[si][1]), si
    mu, sd, theta = plan.stats()
    wmu, wsd, wth = whole_stats
    # the FP32 per-thread partials group other templates (and fundamentals) together,
    # and sigma amplifies that by mu^2 / sigma^2 (up to 8 at stage 8): 1e-7, far
    # inside the 1e-5 the statistics keep against the oracle
    assert np.allclose(mu, wmu, rtol=1e-7, atol=0) and np.allclose(sd, wsd, rtol=1e-7, atol=0)
    assert np.allclose(theta, wth, rtol=1e-6, atol=0)
    got = [(c.stage, c.p, c.t, c.power) for c in plan.candidates()]
    want = [(c.stage, c.p, c.t, c.power) for c in whole_cands]
    if got != want:
        # only a cell at the threshold's last bit may differ
        diff = set(got) ^ set(want)
        stages = list(plan.params.stages)[:ns]
        for (H, p, t, power) in diff:
            si = stages.index(H)
            assert abs(power - float(wth[si])) <= 4e-7 * float(wth[si]), (H, p, power)
    assert len(got) > 0 or not sigma


@pytest.mark.parametrize("mode,stages,thresh,parts", [
    ("sigma", (1, 2), (6.0, 6.0), 1),
    ("abs", (1, 2), (8.0, 11.0), 2),
    ("sigma", (1, 2, 3), (6.0, 6.0, 5.0), 2),
    ("sigma", (1, 2, 4, 8), (5.0, 5.0, 5.0, 5.0), 3),
])
def test_ranges_merged_equal_whole_bank(pkg, mode, stages, thresh, parts):
    from paper_1911_01353_gb300.ranks import template_range
    wl = synth.small_single()
    op = oracle_params(wl, mode=mode, thresh=thresh)
    op.stages = stages
    F = wl.make()
    x = torch.from_numpy(F).cuda()
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        plan.search(x)
        whole_cands = plan.candidates()
        whole_M = [plan.maxproj(si) for si in range(len(stages))]
        whole_stats = plan.stats()
        T = plan.info.n_templates
        split_search(plan, x, [template_range(T, r, parts) for r in range(parts)])
        compare(plan, whole_M, whole_cands, whole_stats, mode == "sigma")
        # the plan searches normally afterwards
        plan.search(x)
        assert [(c.stage, c.p, c.t) for c in plan.candidates()] == [(c.stage, c.p, c.t) for c in whole_cands]


def test_uneven_ranges(pkg):
    """Ranges of very different sizes (one template, a few, the rest) merge to
    the whole search as well."""
    wl = synth.small_single()
    op = oracle_params(wl, mode="sigma", thresh=(6.0, 6.0))
    F = wl.make()
    x = torch.from_numpy(F).cuda()
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        plan.search(x)
        whole_cands = plan.candidates()
        whole_M = [plan.maxproj(si) for si in range(2)]
        whole_stats = plan.stats()
        T = plan.info.n_templates
        split_search(plan, x, [(0, 1), (1, 10), (10, 73), (73, T)])
        compare(plan, whole_M, whole_cands, whole_stats, True)


def test_range_call_order(pkg):
    from paper_1911_01353_gb300 import jerk
    wl = synth.small_single()
    op = oracle_params(wl)
    F = wl.make()
    x = torch.from_numpy(F).cuda()
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        T = plan.info.n_templates
        for lo, hi in ((-1, 5), (5, 5), (0, T + 1), (9, 3)):
            with pytest.raises(jerk.JerkError) as e:
                plan.search_range(x, lo, hi)
            assert e.value.code == jerk.JERK_EINVAL
        plan.search(x)
        with pytest.raises(jerk.JerkError) as e:
            plan.range_sums()                      # the last search was not partial
        assert e.value.code == jerk.JERK_ESTATE
        plan.search_range(x, 0, T // 2)
        with pytest.raises(jerk.JerkError) as e:
            plan.candidates()                      # not selected yet
        assert e.value.code == jerk.JERK_ESTATE
        plan.select()                              # ABS mode: no sums needed
        assert isinstance(plan.candidates(), list)
