"""Pins for the FP64 oracle: every function in ``oracle`` is checked against
something other than itself -- closed forms, library routines (SciPy's
Fresnel integrals and QUADPACK, NumPy's FFT), exact invariants, brute force
on tiny inputs and injected signals with known (r, z, w).

The paper (Adamek et al., Sec. 2-3) prints no worked example, table or
formula, so no pin comes from printed values.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import fresnel

import oracle
import synth


# ---------------------------------------------------------------------------
# The response function rho(q; z, w)
# ---------------------------------------------------------------------------

def test_rho_zero_is_sinc():
    """z = w = 0: the response of an unsmeared sinusoid is sin(pi q)/(pi q)."""
    q = np.array([0.0, 0.25, 0.5, 1.0, 1.5, 2.0, -3.5, 7.25, 40.0])
    got = oracle.rho(q, 0.0, 0.0)
    want = np.sinc(q)
    assert np.max(np.abs(got - want)) < 1e-14
    assert abs(got[2] - 2.0 / math.pi) < 1e-15


def _rho_fresnel(q, z):
    """Closed form for w = 0, z > 0 (completing the square):
    rho = exp(-i pi q^2/z) (2z)^-1/2 [E(s1) - E(s0)],
    s = sqrt(2z) (+-1/2 - q/z), E = C + i S (SciPy's fresnel)."""
    s1 = math.sqrt(2 * z) * (0.5 - q / z)
    s0 = math.sqrt(2 * z) * (-0.5 - q / z)
    S1, C1 = fresnel(s1)
    S0, C0 = fresnel(s0)
    return np.exp(-1j * math.pi * q * q / z) / math.sqrt(2 * z) * ((C1 - C0) + 1j * (S1 - S0))


@pytest.mark.parametrize("q,z", [(0.3, 12.0), (5.5, 40.0), (-3.25, 200.0),
                                 (100.5, 200.0), (-17.0, 2.0), (0.0, 300.0)])
def test_rho_matches_fresnel_closed_form(q, z):
    got = oracle.rho([q], z, 0.0)[0]
    assert abs(got - _rho_fresnel(q, z)) < 1e-12
    # negative z by the conjugate symmetry of the closed form
    got_neg = oracle.rho([q], -z, 0.0)[0]
    assert abs(got_neg - np.conj(_rho_fresnel(-q, z))) < 1e-12


@pytest.mark.parametrize("q,z,w", [(3.3, 30.0, 200.0), (-41.5, -120.0, 560.0),
                                   (0.0, 0.0, 600.0), (150.25, 200.0, -600.0)])
def test_rho_cubic_matches_quadpack(q, z, w):
    """w != 0 has no closed form: compare with SciPy's adaptive QUADPACK."""
    def part(fn):
        return integrate.quad(lambda u: fn(2 * math.pi * (-q * u + z * u * u / 2 + w * u ** 3 / 6)),
                              -0.5, 0.5, limit=4000, epsabs=1e-14, epsrel=1e-13)[0]
    want = part(math.cos) + 1j * part(math.sin)
    got = oracle.rho([q], z, w)[0]
    assert abs(got - want) < 1e-11


def test_rho_conjugate_symmetry():
    q = np.linspace(-30, 30, 121)
    a = oracle.rho(q, 48.0, -340.0)
    b = oracle.rho(-q, -48.0, 340.0)
    assert np.max(np.abs(a - np.conj(b))) < 1e-13


@pytest.mark.parametrize("z,w,delta", [(12.0, 40.0, 0.0), (-80.0, 300.0, 0.5), (0.0, -600.0, 0.25)])
def test_rho_parseval(z, w, delta):
    """sum_n |rho(n + delta)|^2 = 1 (Parseval for the Fourier series of a
    unit-modulus function); the truncated sum misses a 1/q^2 tail."""
    n = np.arange(-1500, 1501, dtype=np.float64)
    s = np.sum(np.abs(oracle.rho(n + delta, z, w)) ** 2)
    assert 0.9995 < s <= 1.0 + 1e-9


def test_rho_quadrature_converged():
    q = np.array([-190.0, -50.5, 0.0, 12.5, 191.0])
    a = oracle.rho(q, 200.0, 600.0)
    b = oracle.rho(q, 200.0, 600.0, panels=4 * (int(191 + 100 + 75) // 4 + 2))
    assert np.max(np.abs(a - b)) < 1e-13


def test_halfwidth_covers_frequency_excursion():
    """m(z, w) - P is the ceiling of max_{|u|<=1/2} |z u + w u^2/2| whenever
    that maximum sits at u = +-1/2, and never below it."""
    assert oracle.halfwidth(20, 60, 16) == 34       # ceil(10 + 7.5) + 16
    assert oracle.halfwidth(200, 600, 16) == 191    # 100 + 75 + 16
    assert oracle.halfwidth(0, 0, 16) == 16
    u = np.linspace(-0.5, 0.5, 20001)
    for z in range(-40, 41, 6):
        for w in range(-200, 201, 40):
            exc = np.max(np.abs(z * u + w * u * u / 2))
            m = oracle.halfwidth(z, w, 0)
            assert m >= exc - 1e-12
            assert m - exc < 1.0 or z * w < 0


# ---------------------------------------------------------------------------
# Correlation
# ---------------------------------------------------------------------------

def test_correlate_bruteforce_tiny():
    rng = np.random.default_rng(5)
    N, b, D = 23, 2, 7
    F = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    c = rng.standard_normal(2 * D + 1) + 1j * rng.standard_normal(2 * D + 1)
    want = np.zeros(b * N, dtype=complex)
    for p in range(b * N):
        for k in range(N):
            d = b * k - p
            if -D <= d <= D:
                want[p] += F[k] * c[d + D]
    got = oracle.correlate(F, c, b)
    assert np.max(np.abs(got - want)) < 1e-13
    got_part = oracle.correlate(F, c, b, p0=9, np_=11)
    assert np.max(np.abs(got_part - want[9:20])) < 1e-13


def test_correlate_equals_fft_overlap_save():
    """Direct correlation = the overlap-and-save FFT route (NumPy FFT), Fig. 1."""
    rng = np.random.default_rng(7)
    N, b = 4096, 2
    F = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    c = oracle.taps(14, -120, b, 16)
    D = (c.size - 1) // 2
    K = c.size
    L = 1024
    V = L - K + 1
    x = np.zeros(b * N + 2 * L, dtype=complex)        # spread, zero-extended
    x[D: D + b * N: b] = F                               # sample j = b k sits at D + j
    g = np.zeros(L, dtype=complex)
    g[:K] = c
    G = np.conj(np.fft.fft(np.conj(g)))                  # sum_m g[m] e^{+2 pi i f m / L}
    out = np.zeros(b * N, dtype=complex)
    for s in range(0, b * N, V):
        seg = x[s: s + L]
        y = np.fft.ifft(np.fft.fft(seg) * G)
        n = min(V, b * N - s)
        out[s: s + n] = y[:n]
    got = oracle.correlate(F, c, b)
    assert np.max(np.abs(got - out)) < 1e-12 * np.max(np.abs(out))


def test_zero_template_integer_cells_are_bin_powers():
    rng = np.random.default_rng(11)
    F = (rng.standard_normal(512) + 1j * rng.standard_normal(512)).astype(np.complex64)
    o = oracle.correlate(F, oracle.taps(0, 0, 2, 16), 2)
    assert np.max(np.abs(np.abs(o[0::2]) ** 2 - np.abs(F.astype(complex)) ** 2)) < 1e-12


def test_zero_template_half_cells_are_interbinning():
    """With one pad bin the z = w = 0 taps sit at q = 0, +-1/2, +-1 and
    rho(+-1) = 0, so half-bin cells give (2/pi)^2 |F_k + F_{k+1}|^2."""
    rng = np.random.default_rng(12)
    F = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    o = oracle.correlate(F, oracle.taps(0, 0, 2, 1), 2)
    want = (2 / math.pi) ** 2 * np.abs(F[:-1] + F[1:]) ** 2
    assert np.max(np.abs(np.abs(o[1:-1:2]) ** 2 - want)) < 1e-12


def test_zero_template_wide_pad_is_fourier_interpolation():
    """With wide padding, half-bin cells approach the exact Fourier
    interpolation (the DFT of the time series at k + 1/2); what is left is the
    truncated sinc tail, bounded for white F by rms|F| (2/(pi^2 P))^1/2."""
    rng = np.random.default_rng(13)
    N = 2048
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    u = (np.arange(N) + 0.5) / N - 0.5
    F = np.array([np.sum(x * np.exp(-2j * np.pi * kk * u)) / N for kk in range(N)])
    k = np.arange(700, 1300)
    half = np.array([np.sum(x * np.exp(-2j * np.pi * (kk + 0.5) * u)) / N for kk in k])
    rms_f = math.sqrt(np.mean(np.abs(F) ** 2))
    errs = []
    for pad in (25, 100, 400):
        o = oracle.correlate(F, oracle.taps(0, 0, 2, pad), 2)
        rms_err = math.sqrt(np.mean(np.abs(o[2 * k + 1] - half) ** 2))
        tail = rms_f * math.sqrt(2.0 / (math.pi ** 2 * pad))
        assert rms_err < 1.5 * tail
        errs.append(rms_err)
    assert errs[0] > errs[1] > errs[2]
    # and it is a real interpolation: far better than the nearest bin
    assert errs[2] < 0.05 * math.sqrt(np.mean(np.abs(F[k] - half) ** 2))


def test_injected_signal_peaks_at_its_cell():
    """Noise-free chirp at (r, z, w) = (10000.25, 12, 40): the (12, 40) template
    is the best at the two neighbouring cells and recovers SNR * sinc(1/4)^2."""
    wl = synth.small_single()
    s = wl.signals[0]
    F = synth.spectrum(wl.n_bins, 1, wl.signals, with_noise=False)
    p = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw)
    bank = oracle.Bank(p)
    zt, wt = oracle.grid(p)
    ts = np.arange(p.n_templates)
    for cell in (20000, 20001):
        pw = bank.power_cells(F, ts, np.full(ts.size, cell))
        t = int(np.argmax(pw))
        assert (zt[t], wt[t]) == (12, 40)
        assert abs(pw[t] - s.snr * np.sinc(0.25) ** 2) < 0.015 * s.snr
    # and the whole-plane max-projection peaks there too
    res = oracle.search(F, oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=(1,),
                                         thresh=(10.0,), norm_block=0), bank)
    assert [(c[0], c[1]) for c in res.candidates] in ([(1, 20000)], [(1, 20001)])


# ---------------------------------------------------------------------------
# Harmonic sums, statistics, peaks
# ---------------------------------------------------------------------------

def test_stage_templates_by_hand():
    p = oracle.Params(20, 2, 60, 20)
    fund, harm = oracle.stage_templates(p, 2)
    zt, wt = oracle.grid(p)
    assert fund.size == 11 * 3          # |z| <= 10 (11 values), |w| <= 30 -> {-20, 0, 20}
    t = int(np.nonzero((zt == 4) & (wt == 20))[0][0])
    row = harm[list(fund).index(t)]
    assert (zt[row[0]], wt[row[0]]) == (4, 20)
    assert (zt[row[1]], wt[row[1]]) == (8, 40)
    fund4, _ = oracle.stage_templates(p, 4)
    assert sorted((int(zt[f]), int(wt[f])) for f in fund4) == [(z, 0) for z in (-4, -2, 0, 2, 4)]


def test_harmonic_sum_recovers_injected_harmonics():
    """A noise-free signal with 2 equal harmonics at (r, z, w) and (2r, 2z, 2w)
    peaks at stage 2 at the fundamental cell and template with S_2 ~ 2 SNR."""
    sig = synth.Signal(5000.0, 4.0, 20.0, 25.0, 0.3)
    F = synth.spectrum(1 << 14, 0, [sig], harmonics=2, with_noise=False)
    p = oracle.Params(20, 2, 60, 20, stages=(1, 2), thresh=(10.0, 30.0), norm_block=0)
    res = oracle.search(F, p)
    zt, wt = oracle.grid(p)
    st2 = [c for c in res.candidates if c[0] == 2]
    assert len(st2) == 1
    H, cell, t, pw = st2[0]
    assert cell == 10000 and (zt[t], wt[t]) == (4, 20)
    assert abs(pw - 2 * sig.snr) < 0.03 * 2 * sig.snr


def test_noise_stats_match_template_energy():
    """Unit white noise: E P = sum over the taps that hit bins of |c_d|^2,
    i.e. half the total tap energy averaged over both cell parities."""
    F = synth.spectrum(1 << 15, 21, ())
    p = oracle.Params(10, 2, 20, 20, stages=(1,), norm_block=0)
    bank = oracle.Bank(p)
    res = oracle.search(F, p, bank)
    mu, sd = res.stats[1]
    energy = np.mean([np.sum(np.abs(bank.taps(t)) ** 2) / 2 for t in range(p.n_templates)])
    assert abs(mu - energy) < 0.01
    assert 0.97 < energy < 1.0
    assert abs(sd - mu) < 0.05                 # exponential power: sd = mean


def test_normalise_is_exact_order_statistic():
    rng = np.random.default_rng(17)
    F = (rng.standard_normal(2500) + 1j * rng.standard_normal(2500)).astype(np.complex64) * 3.0
    out = oracle.normalise(F, 1024)
    for s, e in ((0, 1024), (1024, 2048), (2048, 2500)):
        q = sorted(float(np.float64(a.real) ** 2 + np.float64(a.imag) ** 2) for a in F[s:e])
        med = q[(e - s - 1) // 2]
        scale = 1.0 / math.sqrt(med / math.log(2.0))
        want = (F[s:e].real.astype(np.float64) * scale).astype(np.float32)
        assert np.array_equal(out[s:e].real, want)
    # Exp(1) noise powers come out with unit median -> mean ~ 1
    big = synth.spectrum(1 << 16, 3, ()) * np.float32(7.0)
    pw = np.abs(oracle.normalise(big, 1024).astype(complex)) ** 2
    assert abs(np.median(pw) - math.log(2.0)) < 0.02
    assert abs(np.mean(pw) - 1.0) < 0.02


def test_peak_rules():
    M = np.array([5, 9, 9, 3, 1, 12, 12, 11, 2, 20], dtype=np.float32)
    # 9 at p=1 (plateau keeps lowest p), 12 at p=5, 20 at the right edge
    assert list(oracle.peaks(M, np.float32(4))) == [1, 5, 9]
    assert list(oracle.peaks(M, np.float32(12))) == [9]        # strictly above theta
    assert list(oracle.peaks(np.array([7, 1], np.float32), np.float32(0))) == [0]


def test_maxproj_ties_take_lowest_template():
    S = np.array([[1.0, 3.0, 2.0], [1.0, 3.0, 5.0], [0.5, 1.0, 5.0]])
    M, a = oracle.maxproj(np.array([4, 7, 9]), S)
    assert list(a) == [4, 4, 7] and list(M) == [1.0, 3.0, 5.0]


def test_sigma_threshold_by_hand():
    """SIGMA mode: theta = mu + T sigma with the population statistics."""
    p = oracle.Params(0, 2, 0, 20, stages=(1,), thresh_mode="sigma", thresh=(3.0,))
    S = np.array([[0.0, 2.0, 0.0, 2.0]])          # mu 1, sigma 1
    assert oracle.threshold(p, 0, S) == np.float32(4.0)
    assert oracle.stats(np.array([[1.0, 1.0, 4.0, 6.0]])) == (3.0, math.sqrt(4.5))


# ---------------------------------------------------------------------------
# power at off-grid points (continuous response), refinement, 3-D peaks
# ---------------------------------------------------------------------------

def test_power_at_zero_z_w_is_truncated_sinc_interpolation():
    """z = w = 0: rho(q) = sinc(q), so the response at any r is the classic
    Fourier interpolation sum_k F_k sinc(k - r) over |k - r| <= pad."""
    rng = np.random.default_rng(11)
    F = (rng.standard_normal(300) + 1j * rng.standard_normal(300)) / np.sqrt(2)
    for r in (150.0, 150.5, 150.3, 3.7, 296.2):
        k = np.arange(300)
        sel = np.abs(k - r) <= 16
        A = np.sum(F[sel] * np.sinc(k[sel] - r))
        assert oracle.power_at(F, r, 0.0, 0.0, pad=16) == pytest.approx(abs(A) ** 2, rel=1e-10, abs=1e-12)


def test_power_at_recovers_an_off_grid_chirp():
    """A noiseless signal F_k = A rho(k - r0; z0, w0): by Cauchy-Schwarz the
    response peaks at (r0, z0, w0), where it equals A^2 E^2 with E the energy
    sum_k |rho(k - r0)|^2 of the bins kept (|k - r0| <= m).  Over all k that
    energy is exactly 1 (Poisson summation + Parseval: rho is the transform
    of a unit-modulus function on [-1/2, 1/2]), so E -> 1 as the window grows."""
    r0, z0, w0, A = 200.37, 7.3, 18.6, 3.0
    k = np.arange(400, dtype=np.float64)
    F = A * oracle.rho(k - r0, z0, w0)
    P0 = oracle.power_at(F, r0, z0, w0)
    m = oracle.halfwidth_at(z0, w0, 16)
    kk = k[np.abs(k - r0) <= m]
    E = np.sum(np.abs(oracle.rho(kk - r0, z0, w0)) ** 2)
    assert P0 == pytest.approx(A * A * E * E, rel=1e-9)
    assert 0.99 < E < 1.0
    Ewide = np.sum(np.abs(oracle.rho(k - r0, z0, w0)) ** 2)        # |k - r0| up to ~200 bins
    assert Ewide == pytest.approx(1.0, abs=2e-3) and Ewide > E
    for dr, dz, dw in ((0.1, 0, 0), (-0.1, 0, 0), (0, 0.5, 0), (0, -0.5, 0), (0, 0, 3.0), (0, 0, -3.0),
                       (0.05, 0.2, -1.0)):
        assert oracle.power_at(F, r0 + dr, z0 + dz, w0 + dw) < P0
    (r, z, w, P), c = oracle.refine(F, 200.25, 7.0, 20.0, (0.06, 0.15, 0.7), (3, 3, 3))
    assert abs(r - r0) <= 0.03 and abs(z - z0) <= 0.075 and abs(w - w0) <= 0.35
    assert P >= c


def test_is_peak3d_rules():
    r0, z0, w0 = 100.0, 4.0, 20.0
    k = np.arange(220, dtype=np.float64)
    F = oracle.rho(k - r0, z0, w0)
    assert oracle.is_peak3d(F, r0, z0, w0, 2, 2.0, 20.0)              # the signal's own cell
    assert not oracle.is_peak3d(F, r0 + 0.5, z0, w0, 2, 2.0, 20.0)    # a neighbour is higher
    assert not oracle.is_peak3d(F, r0, z0 + 2.0, w0, 2, 2.0, 20.0)


# ---------------------------------------------------------------------------
# The FFT route (overlap-and-save with the oracle's own radix-2 DFT)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 8, 1024, 8192])
def test_dft_matches_library_fft(n):
    """The oracle's radix-2 DFT against NumPy's FFT (an independent
    implementation), both signs."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    scale = max(1.0, float(np.abs(np.fft.fft(x)).max()))
    assert np.max(np.abs(oracle.dft(x, -1) - np.fft.fft(x))) <= 1e-13 * scale
    assert np.max(np.abs(oracle.dft(x, +1) - np.fft.ifft(x) * n)) <= 1e-13 * scale
    with pytest.raises(ValueError):
        oracle.dft(np.ones(6), -1)


@pytest.mark.parametrize("L", [512, 8192])
def test_fft_route_rows_equal_direct_correlation(L):
    """Every template of a 4096-bin case: the overlap-and-save rows equal the
    direct correlation's |O_p|^2 at every cell to 1e-12 of the row maximum
    (L = 512: 20+ segments with a ragged last one; L = 8192: one segment
    longer than the spread spectrum)."""
    wl = synth.Workload("t", 4096, 20, 2, 60, 20, (1,), (10.0,), 5,
                        [synth.Signal(1000.25, 12.0, 40.0, 40.0, 0.3), synth.Signal(4090.5, -20.0, -60.0, 30.0, 1.0)])
    p = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=(1,))
    Fn = oracle.normalise(wl.make(), p.norm_block)
    bank = oracle.Bank(p)
    rows = oracle.fft_rows(Fn, p, bank, range(p.n_templates), L=L)
    for t in range(p.n_templates):
        o = oracle.correlate(Fn, bank.taps(t), p.numbetween)
        want = o.real * o.real + o.imag * o.imag
        assert np.max(np.abs(rows[t] - want)) <= 1e-12 * want.max(), t


def test_fft_route_rejects_short_transform():
    p = oracle.Params(20, 2, 60, 20, stages=(1,))
    bank = oracle.Bank(p, templates=[0])
    with pytest.raises(ValueError):
        oracle.fft_rows(np.ones(64, np.complex64), p, bank, [0], L=64)      # L below 2 D + 1


@pytest.mark.parametrize("mode,thresh,stages", [("abs", (15.0, 20.0), (1, 2)), ("sigma", (5.0, 5.0, 4.0), (1, 2, 3))])
def test_fft_search_equals_direct_search(mode, thresh, stages):
    """The whole search by the FFT route against ``search`` (direct
    summation, the whole plane held): identical candidates, max-projections
    and argmax (outside exact FP32 ties), runner-up values equal to the
    second-largest FP32 harmonic sum per cell, statistics to 1e-12."""
    wl = synth.small_single()
    p = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=stages, thresh_mode=mode, thresh=thresh)
    F = wl.make()
    ref = oracle.search(F, p)
    got = oracle.fft_search(oracle.normalise(F, p.norm_block), p, L=2048)
    assert got.candidates == ref.candidates and len(ref.candidates) > 0
    for H in stages:
        M, arg = ref.maxproj[H]
        fund, S = ref.sums[H]
        S32 = np.sort(S.astype(np.float32), axis=0)
        assert np.array_equal(got.maxproj[H][0], M)
        assert np.array_equal(got.runner_up[H], S32[-2])
        tie = S32[-1] == S32[-2]
        assert np.array_equal(got.maxproj[H][1][~tie], arg[~tie])
        for a, b in zip(got.stats[H], ref.stats[H]):
            assert abs(a - b) <= 1e-12 * abs(b)
        assert got.theta[H] == ref.theta[H]
    assert got.rows == sum(max(h for h in stages if abs(h * z) <= p.zmax and abs(h * w) <= p.wmax)
                           for z, w in zip(*oracle.grid(p)))


def test_fft_search_reproduces_stored_direct_result():
    """The stored direct-summation result of the 2^16-bin workload
    (tests/golden/small_single_candidates.json, written by make_golden.py
    from ``oracle.search``) is reproduced by the FFT route."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_single_candidates.json")
    with open(path) as f:
        g = json.load(f)
    wl = synth.small_single()
    q = g["params"]
    p = oracle.Params(q["zmax"], q["dz"], q["wmax"], q["dw"], stages=tuple(q["stages"]),
                      thresh_mode=q["thresh_mode"], thresh=tuple(q["thresh"]), norm_block=q["norm_block"])
    got = oracle.fft_search(oracle.normalise(wl.make(), p.norm_block), p)
    assert [list(c) for c in got.candidates] == g["candidates"]
    for H, (mu, sd) in g["stats"].items():
        assert abs(got.stats[int(H)][0] - mu) <= 1e-12 * mu
        assert abs(got.stats[int(H)][1] - sd) <= 1e-12 * sd


def test_fft_search_subset_of_fundamentals():
    """Processing only some fundamentals gives the max over those alone."""
    wl = synth.small_single()
    p = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=(1,))
    Fn = oracle.normalise(wl.make(), p.norm_block)
    sub = [3, 40, 77, 146]
    got = oracle.fft_search(Fn, p, fund=sub)
    bank = oracle.Bank(p, templates=sub)
    P = np.stack([np.abs(oracle.correlate(Fn, bank.taps(t), p.numbetween)) ** 2 for t in sub])
    P32 = P.astype(np.float32)
    assert np.array_equal(got.maxproj[1][0], P32.max(axis=0))
    assert got.rows == len(sub)


def test_power_cells_equal_correlate():
    """Bank.power_cells (its own C loop with per-template offsets) equals
    |correlate|^2 at random (t, p) over templates of different half-widths,
    including cells at both ends of the spectrum."""
    wl = synth.small_single()
    p = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw)
    Fn = oracle.normalise(wl.make(), p.norm_block)
    bN = p.numbetween * Fn.size
    picks = [0, 10, 44, 63, 73, 146]                    # m = 34, 24, 27, 26, 16, 34 bins
    bank = oracle.Bank(p, templates=picks)
    assert len({int(bank.D[t]) for t in picks}) >= 4
    rng = np.random.default_rng(31)
    ps = np.concatenate([[0, 1, 2, 5, bN - 3, bN - 2, bN - 1], rng.integers(0, bN, 200),
                         [20000, 20001]])
    full = {t: np.abs(oracle.correlate(Fn, bank.taps(t), p.numbetween)) ** 2 for t in picks}
    tt = np.repeat(picks, ps.size)
    pp = np.tile(ps, len(picks))
    got = bank.power_cells(Fn, tt, pp)
    want = np.array([full[int(t)][int(q)] for t, q in zip(tt, pp)])
    assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, want.max())


# ---------------------------------------------------------------------------
# The sub-harmonic form (harmonic sum indexed by the highest harmonic)
# ---------------------------------------------------------------------------

def test_round_ratio_by_hand():
    a = np.array([-7, -5, -3, -1, 0, 1, 3, 5, 7])
    assert oracle.round_ratio(a, 1, 2).tolist() == [-4, -3, -2, -1, 0, 1, 2, 3, 4]     # halves away from 0
    assert oracle.round_ratio([10, 11, 12], 1, 3).tolist() == [3, 4, 4]
    assert oracle.round_ratio([10, 11, 12], 2, 3).tolist() == [7, 7, 8]
    assert oracle.round_ratio([9], 5, 8).tolist() == [6]                                # 5.625 -> 6
    assert oracle.round_ratio([-9], 3, 8).tolist() == [-3]                              # -3.375 -> -3


def test_subharmonic_templates_by_hand():
    p = oracle.Params(20, 2, 60, 20)                       # z index -10..10, w index -3..3
    sub = oracle.subharmonic_templates(p, 4)
    t = 6 * 21 + 17                                        # w = +60 (j = 6), z = +14 (i = 17)
    want = []
    for zi, wi in ((2, 1), (4, 2), (5, 2), (7, 3)):         # round(h 7 / 4), round(h 3 / 4), h = 1..4
        want.append((wi + 3) * 21 + zi + 10)
    assert sub[t].tolist() == want
    assert np.array_equal(oracle.subharmonic_templates(p, 1)[:, 0], np.arange(p.n_templates))


@pytest.mark.parametrize("H", [2, 3, 4])
def test_subharmonic_sum_equals_fundamental_sum_where_exact(H):
    """Where the top harmonic sits at (H q, H z, H w) every rounding is exact,
    and the sub-harmonic sum adds the very terms of the fundamental-indexed
    sum S_H(q, z, w), in the same order: the two are bitwise equal there."""
    wl = synth.Workload("t", 3000, 20, 2, 60, 20, (1, H), (10.0, 10.0), 7,
                        [synth.Signal(300.5, 4.0, 20.0, 40.0, 0.2)], harmonics=H)
    p = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=(1, H))
    Fn = oracle.normalise(wl.make(), p.norm_block)
    P = oracle.plane(Fn, p)
    Sp = oracle.subharmonic_sums(P, p, H)
    fund, S = oracle.harmonic_sums(P, p)[H]
    zt, wt = oracle.grid(p)
    for k, f in enumerate(fund):
        top = ((H * wt[f] + p.wmax) // p.dw) * p.nz + (H * zt[f] + p.zmax) // p.dz
        q = np.arange(S.shape[1])
        assert np.array_equal(Sp[top, H * q], S[k])


def test_subharmonic_search_finds_the_top_harmonic():
    """A signal with 4 harmonics of power 30 each, fundamental at
    (r, z, w) = (1000.25, 3, 10): the stage-4 sub-harmonic max-projection
    peaks at the 4th harmonic's cell (r = 4001) with about the sum of the
    four powers there, and stage 1 finds the fundamental."""
    sig = synth.Signal(1000.25, 3.0, 10.0, 30.0, 0.4)
    wl = synth.Workload("t", 1 << 13, 20, 2, 60, 20, (1, 4), (20.0, 60.0), 9, [sig], harmonics=4)
    p = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=(1, 4), thresh=(20.0, 60.0))
    res = oracle.subharmonic_search(wl.make(), p)
    M4, arg4 = res.maxproj[4]
    q = int(np.argmax(M4))
    assert abs(q - 2 * 4 * sig.r) <= 1
    zt, wt = oracle.grid(p)
    assert abs(zt[arg4[q]] - 4 * sig.z) <= 2 and abs(wt[arg4[q]] - 4 * sig.w) <= 20
    assert 0.6 * 4 * sig.snr < M4[q] < 1.2 * 4 * sig.snr + 10
    assert any(H == 4 and abs(c - q) <= 1 for H, c, _, _ in res.candidates)
    M1, _ = res.maxproj[1]
    assert abs(int(np.argmax(M1[:4000])) - 2 * sig.r) <= 1
