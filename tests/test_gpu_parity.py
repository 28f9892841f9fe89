"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes: the 2^16-bin workload (34 segments at L = 4096), ragged spectra that
span many segments with a partial last one, tiny and degenerate inputs.
Tolerance: FP32 powers within 1e-4 of the plane maximum (PLANE_TOL);
integer/index results (medians, candidate cells, templates) exact, with the
guard band documented in ``parity.compare_candidates``.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from parity import (PLANE_TOL, compare_candidates, compare_maxproj, jerk_params, lib_ready,
                    oracle_params)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib_ready()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------------------
# single steps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,block", [(50001, 1024), (4096, 1000), (7, 1024), (1, 16)])
def test_normalise_is_bitwise(pkg, n, block):
    rng = np.random.default_rng(n)
    F = ((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * rng.uniform(0.1, 10, n)).astype(np.complex64)
    op = oracle.Params(4, 2, 0, 20, stages=(1,), thresh=(10.0,), norm_block=block)
    with pkg.Plan(jerk_params(op, n), build_templates=False) as plan:
        x = dev(F)
        y = torch.empty_like(x)
        plan.normalise(x, y)
        got = y.cpu().numpy()
    want = oracle.normalise(F, block)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_normalise_zero_block_is_copied(pkg):
    F = np.zeros(3000, np.complex64)
    F[2500:] = 1 + 1j
    op = oracle.Params(4, 2, 0, 20, stages=(1,), thresh=(10.0,), norm_block=1024)
    with pkg.Plan(jerk_params(op, F.size), build_templates=False) as plan:
        x = dev(F)
        y = torch.empty_like(x)
        plan.normalise(x, y)
        got = y.cpu().numpy()
    assert np.array_equal(got, oracle.normalise(F, 1024))


def _taps_gpu(plan, t0, nt, K):
    out = torch.zeros((nt, K), dtype=torch.complex128, device="cuda")
    plan.taps(t0, nt, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_taps_small_bank(pkg):
    wl = synth.small_single()
    op = oracle_params(wl)
    with pkg.Plan(jerk_params(op, 4096), build_templates=False) as plan:
        K = plan.info.taps
        got = _taps_gpu(plan, 0, op.n_templates, K)
    bank = oracle.Bank(op)
    bM = (K - 1) // 2
    for t in range(op.n_templates):
        c = bank.taps(t)
        D = (c.size - 1) // 2
        want = np.zeros(K, complex)
        want[bM - D: bM + D + 1] = c
        assert np.max(np.abs(got[t] - want)) < 1e-12, t


def test_taps_paper_scale_sample(pkg):
    """zmax 200 / wmax 600 bank: the extreme and a spread of templates."""
    op = oracle.Params(200, 2, 600, 20)
    zt, wt = oracle.grid(op)
    pick = [0, op.n_templates - 1, op.nz - 1, op.n_templates - op.nz, op.n_templates // 2]
    rng = np.random.default_rng(3)
    pick += list(rng.choice(op.n_templates, 7, replace=False))
    with pkg.Plan(jerk_params(op, 4096), build_templates=False) as plan:
        K = plan.info.taps
        assert K == 765
        for t in pick:
            got = _taps_gpu(plan, int(t), 1, K)[0]
            c = oracle.taps(int(zt[t]), int(wt[t]), 2, 16)
            D = (c.size - 1) // 2
            want = np.zeros(K, complex)
            want[382 - D: 382 + D + 1] = c
            assert np.max(np.abs(got - want)) < 1e-11, (t, zt[t], wt[t])


def fold_spectrum(G, L):
    """The folded form the FP32 filter's bank stores: interleaved, the sums of
    the two halves of G and their differences times exp(+2 pi i k / R0), k
    the element's DFT index in the first inverse pass of radix R0."""
    log2L = int(round(np.log2(L)))
    R0 = 1 << (log2L % 4) if log2L % 4 else 16
    NT, I0, h = L // 16, 16 // R0, L // 2
    f = np.arange(h)
    k = (f // NT) // I0
    out = np.empty(L, dtype=complex)
    out[0::2] = G[:h] + G[h:]
    out[1::2] = (G[:h] - G[h:]) * np.exp(2j * np.pi * k / R0)
    return out


def pair_spectrum(G, P):
    """The paired form the tensor-core filter's bank stores: values f and
    f + P (bit log2 P of f clear) side by side, real parts then imaginary
    parts, as two complex64 slots per pair."""
    f = np.arange(G.size)
    f = f[(f & P) == 0]
    out = np.empty(G.size, dtype=complex)
    out[0::2] = G[f].real + 1j * G[f + P].real
    out[1::2] = G[f].imag + 1j * G[f + P].imag
    return out


@pytest.mark.parametrize("precision,seg_len", [(0, 0), (0, 2048), (0, 8192), (2, 0)])
def test_bank_spectra(pkg, precision, seg_len):
    """Stored FP32 template spectra = (1/L) sum_m g[m] e^{+2 pi i f m / L} of the
    oracle's taps (NumPy FFT), to FP32 rounding: in the paired form for the
    tensor-core filters, in the folded form for the FP32 filter."""
    wl = synth.small_single()
    op = oracle_params(wl)
    p = jerk_params(op, 1 << 16, seg_len=seg_len)
    p.precision = precision
    with pkg.Plan(p) as plan:
        L, K, T = plan.info.seg_len, plan.info.taps, plan.info.n_templates
        torch.cuda.synchronize()
        from paper_1911_01353_gb300.jerk import _DevArray
        bank = torch.as_tensor(_DevArray(plan.info.d_bank, T * L * 2, "<f4"), device="cuda").cpu().numpy()
        bank = bank.view(np.complex64).reshape(T, L)
        plan_rows = {t: plan.template_row(t) for t in range(T)}
        assert sorted(r for r, _, _ in plan_rows.values()) == list(range(T))
    ob = oracle.Bank(op)
    rows = set()
    for t in (0, 17, 73, 100, T - 1):
        row, bMg, Vg = plan_rows[t]
        rows.add(row)
        assert Vg == L - 2 * bMg and bMg >= 2 * oracle.halfwidth(int(ob.zt[t]), int(ob.wt[t]), 16)
        c = ob.taps(t)
        D = (c.size - 1) // 2
        g = np.zeros(L, complex)
        g[bMg - D: bMg + D + 1] = c
        want = np.fft.ifft(g)          # (1/L) sum_m g[m] e^{+2 pi i f m / L}
        if precision == 0:
            want = fold_spectrum(want, L)
        else:
            want = pair_spectrum(want, 64)
        assert np.max(np.abs(bank[row] - want)) < 2e-7 * np.max(np.abs(want)) + 1e-9
    assert len(rows) == 5


# ---------------------------------------------------------------------------
# the power plane
# ---------------------------------------------------------------------------

def _plane_gpu(plan, F, t0, nt):
    x = dev(F)
    out = torch.empty((nt, 2 * F.size), dtype=torch.float32, device="cuda")
    plan.plane(x, t0, nt, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def small(pkg):
    wl = synth.small_single()
    op = oracle_params(wl)
    F = wl.make()
    res = oracle.search(F, op, keep_plane=True)
    return wl, op, F, res


def test_plane_small(pkg, small):
    wl, op, F, res = small
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        got = _plane_gpu(plan, F, 0, op.n_templates)
    want = res.plane
    tol = PLANE_TOL * want.max()
    err = np.abs(got - want)
    assert err.max() <= tol, (err.max(), tol)
    # far tighter in practice; record the scale of the error
    assert err.max() <= 1e-5 * want.max()


@pytest.mark.parametrize("seg_len", [1024, 2048, 8192])
def test_plane_ragged_tiles(pkg, seg_len):
    """50001 bins: many segments and a partial last one, for each L."""
    n = 50001
    sig = synth.Signal(12345.5, -6.0, 20.0, 40.0, 1.0)
    F = synth.spectrum(n, 9, [sig])
    op = oracle.Params(10, 2, 40, 20, stages=(1,), thresh=(12.0,))
    with pkg.Plan(jerk_params(op, n, seg_len=seg_len)) as plan:
        assert plan.info.seg_len == seg_len
        got = _plane_gpu(plan, F, 3, 9)
    want = oracle.plane(oracle.normalise(F, 1024), op)[3:12]
    assert np.max(np.abs(got - want)) <= PLANE_TOL * want.max()


# ---------------------------------------------------------------------------
# the whole path
# ---------------------------------------------------------------------------

def _search(pkg, plan, F, host=False):
    if host:
        plan.search_host(F)
    else:
        x = dev(F)
        plan.search(x)
    return plan.candidates()


def test_search_small(pkg, small):
    wl, op, F, res = small
    tol = PLANE_TOL * res.plane.max()
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        cands = _search(pkg, plan, F)
        for si, H in enumerate(op.stages):
            M, t = plan.maxproj(si)
            Mo, to = res.maxproj[H]
            fund, S = res.sums[H]
            compare_maxproj(M, t, Mo, to, S, tol)
    guarded = compare_candidates(cands, res, tol)
    assert guarded <= 2
    # the injected chirp at r = 10000.25 is found at stage 1 within half a bin
    assert any(c.stage == 1 and abs(c.r - 10000.25) <= 0.25 for c in cands)


@pytest.mark.parametrize("group_size", [1, 7, 64])
def test_search_small_tile_shapes(pkg, small, group_size):
    """Other template-group sizes (the autotuner's tile-shape parameter): one
    template per group, a group size that leaves ragged groups, larger groups;
    every stage and the candidates against the oracle as in test_search_small."""
    wl, op, F, res = small
    tol = PLANE_TOL * res.plane.max()
    p = jerk_params(op, F.size)
    p.group_size = group_size
    with pkg.Plan(p) as plan:
        assert plan.info.n_groups == -(-op.n_templates // group_size)
        cands = _search(pkg, plan, F)
        for si, H in enumerate(op.stages):
            M, t = plan.maxproj(si)
            compare_maxproj(M, t, res.maxproj[H][0], res.maxproj[H][1], res.sums[H][1], tol)
    assert compare_candidates(cands, res, tol) <= 2


def _dropped_outputs(op, seg_len, group_size):
    """Per template group (sorted by half-width, runs of group_size), the
    number of last-pass outputs r that every thread drops: 16 - ceil(V / NT),
    V = L - 4 max m (interbinning b = 2), at most 2."""
    nz = 2 * op.zmax // op.dz + 1
    nw = 2 * op.wmax // op.dw + 1
    m = [oracle.halfwidth(-op.zmax + (t % nz) * op.dz, -op.wmax + (t // nz) * op.dw, op.pad_bins)
         for t in range(nz * nw)]
    order = sorted(range(nz * nw), key=lambda t: (m[t], t))
    nt = seg_len // 16
    out = set()
    for k0 in range(0, len(order), group_size):
        V = seg_len - 4 * max(m[t] for t in order[k0:k0 + group_size])
        out.add(min(2, 16 - -(-V // nt)))
    return out


@pytest.mark.parametrize("seg_len,group_size,drops", [(1024, 16, {1, 2}), (2048, 16, {0, 1}),
                                                       (4096, 16, {0})])
def test_search_small_dropped_outputs(pkg, small, seg_len, group_size, drops):
    """The filter skips the last-pass outputs that lie in every segment's
    overlap (0, 1 or 2 per thread by template group): search mode at segment
    lengths and group sizes that give each count, every stage, the SIGMA
    statistics and the candidates against the oracle."""
    wl, _, F, _ = small
    op = oracle_params(wl, mode="sigma", thresh=(13.0, 12.0))
    assert _dropped_outputs(op, seg_len, group_size) == drops
    res = oracle.search(F, op)
    tol = PLANE_TOL * max(float(res.maxproj[H][0].max()) for H in op.stages)
    p = jerk_params(op, F.size, seg_len=seg_len)
    p.group_size = group_size
    with pkg.Plan(p) as plan:
        assert plan.info.seg_len == seg_len
        cands = _search(pkg, plan, F)
        mu, sd, _ = plan.stats()
        for si, H in enumerate(op.stages):
            M, t = plan.maxproj(si)
            compare_maxproj(M, t, res.maxproj[H][0], res.maxproj[H][1], res.sums[H][1], tol)
            assert abs(mu[si] - res.stats[H][0]) <= 1e-5 * res.stats[H][0]
            assert abs(sd[si] - res.stats[H][1]) <= 1e-5 * res.stats[H][1]
    assert compare_candidates(cands, res, tol) <= 2


def test_search_small_sigma_mode(pkg, small):
    wl, op0, F, _ = small
    op = oracle_params(wl, mode="sigma", thresh=(13.0, 12.0))
    res = oracle.search(F, op)
    tol = PLANE_TOL * max(float(res.maxproj[H][0].max()) for H in op.stages)
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        cands = _search(pkg, plan, F)
        mu, sd, th = plan.stats()
    for si, H in enumerate(op.stages):
        assert abs(mu[si] - res.stats[H][0]) <= 1e-5 * res.stats[H][0]
        assert abs(sd[si] - res.stats[H][1]) <= 1e-5 * res.stats[H][1]
        assert abs(th[si] - float(res.theta[H])) <= 1e-5 * float(res.theta[H])
    compare_candidates(cands, res, tol)


def test_search_host_equals_device(pkg, small):
    wl, op, F, res = small
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        a = [(c.stage, c.p, c.t, c.power) for c in _search(pkg, plan, F)]
        b = [(c.stage, c.p, c.t, c.power) for c in _search(pkg, plan, F, host=True)]
        c2 = [(c.stage, c.p, c.t, c.power) for c in _search(pkg, plan, F)]
    assert a == b == c2          # bitwise repeatable


def test_harmonic_stages_1_2_4_8(pkg):
    """Four stages on a signal with 8 harmonics: every stage vs the oracle."""
    n = 1 << 15
    sig = synth.Signal(3000.0, 2.0, 20.0, 6.0, 0.4)
    F = synth.spectrum(n, 31, [sig], harmonics=8)
    op = oracle.Params(16, 2, 160, 20, stages=(1, 2, 4, 8), thresh=(12.0, 18.0, 26.0, 40.0))
    res = oracle.search(F, op, keep_plane=True)
    tol = PLANE_TOL * res.plane.max()
    with pkg.Plan(jerk_params(op, n)) as plan:
        cands = _search(pkg, plan, F)
        for si, H in enumerate(op.stages):
            M, t = plan.maxproj(si)
            Mo, to = res.maxproj[H]
            compare_maxproj(M, t, Mo, to, res.sums[H][1], tol)
    compare_candidates(cands, res, tol)
    st8 = [c for c in cands if c.stage == 8]
    assert any(c.p == 6000 and (c.z, c.w) == (2.0, 20.0) for c in st8)


@pytest.mark.parametrize("stages", [(1,), (1, 3), (1, 2, 3, 5)])
def test_other_stage_sets(pkg, stages):
    n = 20000
    F = synth.spectrum(n, 41, [synth.Signal(2500.5, 4.0, 0.0, 30.0, 0.0)], harmonics=5)
    th = (10.0, 14.0, 18.0, 22.0)[:len(stages)]
    op = oracle.Params(8, 2, 20, 10, stages=stages, thresh=th)
    res = oracle.search(F, op, keep_plane=True)
    tol = PLANE_TOL * res.plane.max()
    with pkg.Plan(jerk_params(op, n, seg_len=1024)) as plan:
        cands = _search(pkg, plan, F)
        for si, H in enumerate(stages):
            M, t = plan.maxproj(si)
            compare_maxproj(M, t, *res.maxproj[H], res.sums[H][1], tol)
    compare_candidates(cands, res, tol)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("zmax,wmax,stages", [(0, 0, (1, 2, 4, 8)), (0, 20, (1, 2)), (2, 0, (1, 2, 4)),
                                              (2, 20, (1, 2, 3))])
def test_degenerate_banks(pkg, zmax, wmax, stages):
    """Banks of 1 to 9 templates: template groups of one or two (the ends of
    the per-template metadata pipeline) and, for z = w = 0, one template that
    is its own h-th harmonic for every h up to 8 (the most harmonic-row
    entries a template can have).  Every stage and the candidates vs the
    oracle."""
    n = 12000
    F = synth.spectrum(n, 53, [synth.Signal(1000.0, 0.0, 0.0, 25.0, 0.3)], harmonics=8)
    th = (10.0, 14.0, 18.0, 26.0)[:len(stages)]
    op = oracle.Params(zmax, 2, wmax, 20, stages=stages, thresh=th)
    res = oracle.search(F, op, keep_plane=True)
    tol = PLANE_TOL * res.plane.max()
    with pkg.Plan(jerk_params(op, n, seg_len=1024)) as plan:
        assert plan.info.n_templates == op.n_templates
        cands = _search(pkg, plan, F)
        for si, H in enumerate(stages):
            M, t = plan.maxproj(si)
            compare_maxproj(M, t, *res.maxproj[H], res.sums[H][1], tol)
    compare_candidates(cands, res, tol)
    assert any(c.stage == stages[-1] and c.p == 2000 for c in cands)


@pytest.mark.parametrize("n", [1, 2, 3, 1023, 1025])
def test_tiny_spectra(pkg, n):
    rng = np.random.default_rng(n + 100)
    F = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64) * 3
    op = oracle.Params(4, 2, 20, 20, stages=(1, 2), thresh=(0.5, 1.0))
    res = oracle.search(F, op, keep_plane=True)
    tol = PLANE_TOL * max(res.plane.max(), 1e-30)
    with pkg.Plan(jerk_params(op, 2048, seg_len=1024)) as plan:
        cands = _search(pkg, plan, F)
        for si, H in enumerate(op.stages):
            M, t = plan.maxproj(si)
            compare_maxproj(M, t, *res.maxproj[H], res.sums[H][1], tol)
    compare_candidates(cands, res, tol)


def test_zero_spectrum_has_no_candidates(pkg):
    F = np.zeros(4096, np.complex64)
    op = oracle.Params(10, 2, 20, 20, stages=(1, 2), thresh=(1e-3, 1e-3))
    with pkg.Plan(jerk_params(op, 4096)) as plan:
        assert _search(pkg, plan, F) == []
        M, t = plan.maxproj(0)
        assert np.all(M == 0) and np.all(t == 0)


def test_full_capacity_and_reuse(pkg):
    """A spectrum of exactly max_bins, then a shorter one on the same plan."""
    op = oracle.Params(6, 2, 20, 20, stages=(1, 2), thresh=(9.0, 12.0))
    with pkg.Plan(jerk_params(op, 30000, seg_len=2048)) as plan:
        for n, seed in ((30000, 51), (12345, 52)):
            F = synth.spectrum(n, seed, [synth.Signal(n / 3 + 0.5, 2.0, 20.0, 25.0, 0.1)])
            res = oracle.search(F, op, keep_plane=True)
            tol = PLANE_TOL * res.plane.max()
            cands = _search(pkg, plan, F)
            for si, H in enumerate(op.stages):
                M, t = plan.maxproj(si)
                compare_maxproj(M, t, *res.maxproj[H], res.sums[H][1], tol)
            compare_candidates(cands, res, tol)


def test_call_order_and_bounds(pkg):
    from paper_1911_01353_gb300 import jerk
    op = oracle.Params(4, 2, 0, 20, stages=(1,), thresh=(5.0,))
    with pkg.Plan(jerk_params(op, 1000), build_templates=False) as plan:
        x = dev(np.ones(1000, np.complex64))
        with pytest.raises(jerk.JerkError) as e:
            plan.search(x)
        assert e.value.code == jerk.JERK_ESTATE
        plan.templates()
        with pytest.raises(jerk.JerkError) as e:
            plan.search(dev(np.ones(1001, np.complex64)))
        assert e.value.code == jerk.JERK_EINVAL


def test_candidate_overflow_reports_true_count(pkg):
    from paper_1911_01353_gb300 import jerk
    n = 8192
    F = synth.spectrum(n, 61, ())
    op = oracle.Params(4, 2, 0, 20, stages=(1,), thresh=(0.0,))
    with pkg.Plan(jerk_params(op, n, max_candidates=16)) as plan:
        plan.search(dev(F))
        with pytest.raises(jerk.JerkError) as e:
            plan.candidates()
        assert e.value.code == jerk.JERK_EOVERFLOW
    res = oracle.search(F, op)
    assert len(res.candidates) > 16


# ---------------------------------------------------------------------------
# roofline denominators
# ---------------------------------------------------------------------------

def test_packed_fma_rate_equals_scalar(pkg):
    """Packed (f32x2) FMAs run at the scalar FMA rate: the filters use them to
    save issue slots, and their FP32 roofline keeps the scalar peak as its
    denominator.  A packed rate near twice the scalar one would make that
    denominator wrong, and this test fails then."""
    f32, l2 = pkg.measure_peaks(0)
    f32x2 = pkg.measure_packed_fma(0)
    assert f32 > 0 and l2 > 0 and f32x2 > 0
    assert 0.8 < f32x2 / f32 < 1.25, (f32, f32x2)
