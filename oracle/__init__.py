"""FP64 CPU oracle for the Fourier-domain jerk search.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The CUDA path never calls it, and it never calls the CUDA path: the two
share no code, headers, tables or constants.  Inputs come from ``synth``.

What it computes, in the order of the paper's pipeline (Adamek et al.,
"Searching for pulsars in extreme orbits", Sec. 2 and Sec. 3):

1. ``normalise``      power normalisation of the spectrum (the paper is
                      silent; reading: blocks of B bins, lower median of
                      |F|^2, scale (median/ln 2)^-1/2).
2. ``rho`` / ``taps`` the matched filter for each (z, w), z = fdot T^2,
                      w = fddot T^3 (Sec. 2), as the exact Fourier response
                      integral, by quadrature.
3. ``correlate``      the filter applied to the spectrum by direct summation
                      (what overlap-and-save computes, Fig. 1).
4. ``plane``          |.|^2 over (w, z, r).
5. ``harmonic_sums``  S_H(p, z, w) = sum_{h=1..H} P(h p, h z, h w)
                      (Sec. 3 names the harmonic sum; the h set 1..H is a reading).
6. ``stats``          mean and standard deviation of S_H (Sec. 3).
7. ``peaks``          thresholded peak finding on the max-projection over
                      (z, w) (Sec. 3 "peak-finding ... above some user
                      specified threshold"; the 1-D peak rule is a reading).
8. ``fft_search``     steps 3-7 for the whole bank by the FFT route:
                      overlap-and-save with a radix-2 FP64 DFT (``dft``),
                      one power row at a time, never the whole plane; the
                      harmonic sums, max-projections (with the runner-up
                      value per cell) and statistics accumulated as rows
                      come.  For spectra too long for direct summation.
9. ``power_at``       the filter response at any point (r, z, w) of the
                      continuous parameter space (the plane off its grid),
                      by direct summation with rho; ``refine`` takes its
                      maximum over a small grid around a candidate, and
                      ``is_peak3d`` compares a cell with its 26 neighbours.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, library routines, invariants or brute force.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jerk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libjerk_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (plain FP64, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_rho.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                   dp, dp, ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_correlate.argtypes = [dp, ctypes.c_int64, ctypes.c_int, dp, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int64, dp]
        lib.oracle_power_cells.argtypes = [dp, ctypes.c_int64, ctypes.c_int, dp, lp, lp, lp,
                                           lp, ctypes.c_int64, dp]
        lib.oracle_threads.restype = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int32)
        fp = ctypes.POINTER(ctypes.c_float)
        lib.oracle_dft.argtypes = [dp, ctypes.c_int64, ctypes.c_int]
        lib.oracle_dft.restype = ctypes.c_int
        lib.oracle_fft_search.argtypes = [dp, ctypes.c_int64, ctypes.c_int, dp, lp, lp, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_int, ip, lp, ip, lp, ctypes.c_int64,
                                          lp, fp, ip, fp, dp, lp]
        lib.oracle_fft_search.restype = ctypes.c_int
        lib.oracle_fft_rows.argtypes = [dp, ctypes.c_int64, ctypes.c_int, dp, lp, lp, ctypes.c_int64,
                                        ctypes.c_int64, lp, ctypes.c_int64, dp]
        lib.oracle_fft_rows.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def threads() -> int:
    """OpenMP threads the oracle's C loops use."""
    return int(_load().oracle_threads())


# ---------------------------------------------------------------------------
# Parameters and the (z, w) grid
# ---------------------------------------------------------------------------

@dataclass
class Params:
    """Search parameters (integer grid, as the bank is defined on it)."""
    zmax: int
    dz: int
    wmax: int
    dw: int
    numbetween: int = 2          # b: Fourier cells per bin (interbinning)
    pad_bins: int = 16           # P: extra half-width of every template
    stages: tuple = (1, 2)
    thresh_mode: str = "abs"     # "abs" or "sigma"
    thresh: tuple = (15.0, 20.0)
    norm_block: int = 1024       # B; 0 disables normalisation

    @property
    def nz(self) -> int:
        return 2 * self.zmax // self.dz + 1

    @property
    def nw(self) -> int:
        return 2 * self.wmax // self.dw + 1

    @property
    def n_templates(self) -> int:
        return self.nz * self.nw


def grid(p: Params):
    """(z_t, w_t) for t = j*nz + i, z_i = -zmax + i dz, w_j = -wmax + j dw."""
    z = np.array([-p.zmax + i * p.dz for i in range(p.nz)], dtype=np.int64)
    w = np.array([-p.wmax + j * p.dw for j in range(p.nw)], dtype=np.int64)
    zt = np.tile(z, p.nw)
    wt = np.repeat(w, p.nz)
    return zt, wt


def halfwidth(z: int, w: int, pad: int) -> int:
    """m(z, w) = ceil(|z|/2 + |w|/8) + P bins: the largest excursion of the
    instantaneous frequency r + z u + w u^2/2 over |u| <= 1/2, plus padding
    for the sinc wings (reading: the paper gives no template length)."""
    return (4 * abs(int(z)) + abs(int(w)) + 7) // 8 + int(pad)


# ---------------------------------------------------------------------------
# 2. The response function and the taps
# ---------------------------------------------------------------------------

_GL_N = 32


def _gl():
    x, wt = np.polynomial.legendre.leggauss(_GL_N)
    return np.ascontiguousarray(x), np.ascontiguousarray(wt)


def rho(q, z: float, w: float, panels: int | None = None) -> np.ndarray:
    """rho(q; z, w) = int_{-1/2}^{1/2} exp(2 pi i (-q u + z u^2/2 + w u^3/6)) du.

    The Fourier response, at frequency offset q bins, of a unit signal whose
    frequency, fdot T^2 and fddot T^3 at mid-observation are (r, z, w)
    (Sec. 2 defines z and w; the mid-observation origin is a reading).
    Composite 32-node Gauss-Legendre, with at most 4 cycles of the integrand
    per panel unless ``panels`` is given.
    """
    q = np.ascontiguousarray(np.atleast_1d(np.asarray(q, dtype=np.float64)))
    if panels is None:
        osc = float(np.max(np.abs(q))) + abs(z) / 2.0 + abs(w) / 8.0
        panels = int(math.ceil(osc / 4.0)) + 2
    x, wt = _gl()
    out = np.empty(2 * q.size, dtype=np.float64)
    _load().oracle_rho(_dp(q), q.size, float(z), float(w), _dp(x), _dp(wt), _GL_N,
                       int(panels), _dp(out))
    return out[0::2] + 1j * out[1::2]


def taps(z: int, w: int, b: int, pad: int) -> np.ndarray:
    """c_d = conj(rho(d/b; z, w)) for d = -b m .. b m (index d + b m)."""
    m = halfwidth(z, w, pad)
    d = np.arange(-b * m, b * m + 1, dtype=np.float64)
    return np.conj(rho(d / b, z, w))


# ---------------------------------------------------------------------------
# 1. Normalisation
# ---------------------------------------------------------------------------

LN2 = math.log(2.0)


def normalise(F: np.ndarray, block: int) -> np.ndarray:
    """Power normalisation (reading; the paper is silent).

    For each block of ``block`` bins (the last may be short): q_k = |F_k|^2
    in FP64, med = the element of rank floor((n-1)/2) of the sorted q, and
    F_k <- F_k * (med / ln 2)^(-1/2) (so Exp(1)-distributed noise power has
    unit mean).  A block whose median is 0 is left unscaled.  complex64 out.
    """
    F = np.asarray(F, dtype=np.complex64)
    if block <= 0:
        return F.copy()
    re = F.real.astype(np.float64)
    im = F.imag.astype(np.float64)
    q = re * re + im * im
    ore = np.empty_like(re)
    oim = np.empty_like(im)
    for s in range(0, F.size, block):
        e = min(s + block, F.size)
        blk = np.sort(q[s:e])
        med = blk[(e - s - 1) // 2]
        scale = 1.0 / math.sqrt(med / LN2) if med > 0.0 else 1.0
        ore[s:e] = re[s:e] * scale
        oim[s:e] = im[s:e] * scale
    return (ore.astype(np.float32) + 1j * oim.astype(np.float32)).astype(np.complex64)


# ---------------------------------------------------------------------------
# 3-4. Correlation and power
# ---------------------------------------------------------------------------

def correlate(F: np.ndarray, c: np.ndarray, b: int, p0: int = 0, np_: int | None = None):
    """O_p = sum_k F_k c_{b k - p} over |b k - p| <= D (c has 2D+1 taps),
    bins outside [0, N) being zero; p = p0 .. p0+np-1 (default all b N)."""
    F = np.ascontiguousarray(np.asarray(F, dtype=np.complex128))
    c = np.ascontiguousarray(np.asarray(c, dtype=np.complex128))
    N = F.size
    D = (c.size - 1) // 2
    if np_ is None:
        np_ = b * N - p0
    Fi = F.view(np.float64)
    ci = c.view(np.float64)
    out = np.empty(2 * np_, dtype=np.float64)
    _load().oracle_correlate(_dp(Fi), N, b, _dp(ci), D, p0, np_, _dp(out))
    return out[0::2] + 1j * out[1::2]


class Bank:
    """All templates of a parameter set: taps per template, flattened."""

    def __init__(self, p: Params, templates=None):
        self.p = p
        self.zt, self.wt = grid(p)
        T = p.n_templates
        sel = range(T) if templates is None else templates
        self.D = np.zeros(T, dtype=np.int64)
        self.off = np.zeros(T, dtype=np.int64)
        chunks = []
        pos = 0
        for t in range(T):
            self.D[t] = p.numbetween * halfwidth(self.zt[t], self.wt[t], p.pad_bins)
        for t in sel:
            c = taps(int(self.zt[t]), int(self.wt[t]), p.numbetween, p.pad_bins)
            self.off[t] = pos
            pos += c.size
            chunks.append(c)
        self.flat = np.ascontiguousarray(np.concatenate(chunks)) if chunks else np.zeros(1, complex)

    def taps(self, t: int) -> np.ndarray:
        n = 2 * int(self.D[t]) + 1
        return self.flat[self.off[t]: self.off[t] + n]

    def power_cells(self, Fn: np.ndarray, cell_t, cell_p) -> np.ndarray:
        """|O_p(t)|^2 at explicit (t, p) pairs, by direct correlation."""
        F = np.ascontiguousarray(np.asarray(Fn, dtype=np.complex128))
        ct = np.ascontiguousarray(np.asarray(cell_t, dtype=np.int64))
        cp = np.ascontiguousarray(np.asarray(cell_p, dtype=np.int64))
        out = np.empty(ct.size, dtype=np.float64)
        _load().oracle_power_cells(_dp(F.view(np.float64)), F.size, self.p.numbetween,
                                   _dp(self.flat.view(np.float64)), _lp(self.off), _lp(self.D),
                                   _lp(ct), _lp(cp), ct.size, _dp(out))
        return out


def plane(Fn: np.ndarray, p: Params, bank: Bank | None = None) -> np.ndarray:
    """P[t, p] = |O_p(z_t, w_t)|^2 for every template and every cell (FP64)."""
    bank = bank or Bank(p)
    bN = p.numbetween * Fn.size
    out = np.empty((p.n_templates, bN), dtype=np.float64)
    for t in range(p.n_templates):
        o = correlate(Fn, bank.taps(t), p.numbetween)
        out[t] = o.real * o.real + o.imag * o.imag
    return out


# ---------------------------------------------------------------------------
# 5. Harmonic sums
# ---------------------------------------------------------------------------

def stage_templates(p: Params, H: int):
    """Templates valid as fundamentals at stage H (|H z| <= zmax and
    |H w| <= wmax) and, for each, the template index of (h z, h w), h=1..H."""
    zt, wt = grid(p)
    where = {(int(zt[t]), int(wt[t])): t for t in range(zt.size)}
    fund, harm = [], []
    for t in range(zt.size):
        z, w = int(zt[t]), int(wt[t])
        if abs(H * z) <= p.zmax and abs(H * w) <= p.wmax:
            fund.append(t)
            harm.append([where[(h * z, h * w)] for h in range(1, H + 1)])
    return np.array(fund, dtype=np.int64), np.array(harm, dtype=np.int64).reshape(len(fund), H)


def n_valid(bN: int, H: int) -> int:
    """Number of fundamental cells p with H p < bN."""
    return (bN - 1) // H + 1


def harmonic_sums(P: np.ndarray, p: Params):
    """{H: (fund, S_H)} with S_H[f, p] = sum_{h=1..H} P[t_h(f), h p] for the
    valid fundamentals f and cells p < n_valid(bN, H); sums in FP64 in h order."""
    bN = P.shape[1]
    out = {}
    for H in p.stages:
        fund, harm = stage_templates(p, H)
        n = n_valid(bN, H)
        S = np.zeros((fund.size, n), dtype=np.float64)
        pp = np.arange(n)
        for h in range(1, H + 1):
            S += P[harm[:, h - 1]][:, h * pp]
        out[H] = (fund, S)
    return out


# ---------------------------------------------------------------------------
# 6-7. Statistics, max-projection, thresholds and peaks
# ---------------------------------------------------------------------------

def stats(S: np.ndarray):
    """Population mean and standard deviation of all cells of S_H (FP64)."""
    mu = float(np.mean(S))
    sd = float(np.sqrt(np.mean((S - mu) ** 2)))
    return mu, sd


def maxproj(fund: np.ndarray, S: np.ndarray):
    """M_H(p) = max_f S_H[f, p] rounded to FP32 (decisions are taken in the
    kernel's precision), argmax = lowest template index among equal FP32
    values.  ``fund`` is sorted ascending so the first maximum is the lowest t."""
    S32 = S.astype(np.float32)
    a = np.argmax(S32, axis=0)
    return S32[a, np.arange(S.shape[1])], fund[a]


def threshold(p: Params, si: int, S: np.ndarray | None = None) -> np.float32:
    """theta_H: ABS mode -> the given power; SIGMA mode -> mu + T sigma."""
    T = p.thresh[si]
    if p.thresh_mode == "abs":
        return np.float32(T)
    mu, sd = stats(S)
    return np.float32(mu + T * sd)


def peaks(M: np.ndarray, theta: np.float32) -> np.ndarray:
    """Cells p with M(p) > theta, M(p) > M(p-1) and M(p) >= M(p+1); a
    missing neighbour counts as -inf (reading of Sec. 3's peak finding:
    1-D local maxima along r of the (z, w) max-projection; a plateau keeps
    its lowest p)."""
    M = np.asarray(M, dtype=np.float32)
    left = np.concatenate([[-np.inf], M[:-1]]).astype(np.float64)
    right = np.concatenate([M[1:], [-np.inf]]).astype(np.float64)
    m = M.astype(np.float64)
    ok = (m > float(theta)) & (m > left) & (m >= right)
    return np.nonzero(ok)[0]


@dataclass
class Result:
    candidates: list = field(default_factory=list)   # (stage, p, t, power32)
    maxproj: dict = field(default_factory=dict)      # H -> (M float32, argmax t)
    theta: dict = field(default_factory=dict)        # H -> float32
    stats: dict = field(default_factory=dict)        # H -> (mu, sd)
    sums: dict = field(default_factory=dict)         # H -> (fund, S_H fp64)


def halfwidth_at(z: float, w: float, pad: int) -> int:
    """m(z, w) = ceil(|z|/2 + |w|/8) + P for real z, w (equal to
    ``halfwidth`` on the integer grid)."""
    return int(math.ceil(abs(z) / 2.0 + abs(w) / 8.0)) + int(pad)


def power_at(Fn: np.ndarray, r: float, z: float, w: float, pad: int = 16) -> float:
    """P(r, z, w) = |sum_k Fn_k conj(rho(k - r; z, w))|^2 over the bins
    |k - r| <= m(z, w), bins outside [0, N) being zero: the matched-filter
    power of Sec. 2 at any point of the continuous (r, z, w) space.  On the
    grid (r = p / b, integer z, w) it is the plane value P(p, z, w), since
    the taps are c_d = conj(rho(d/b)) with d = b k - p."""
    Fn = np.asarray(Fn)
    m = halfwidth_at(z, w, pad)
    k0 = max(0, int(math.ceil(r - m)))
    k1 = min(Fn.size - 1, int(math.floor(r + m)))
    if k1 < k0:
        return 0.0
    k = np.arange(k0, k1 + 1, dtype=np.float64)
    A = np.sum(Fn[k0:k1 + 1].astype(np.complex128) * np.conj(rho(k - r, z, w)))
    return float(A.real * A.real + A.imag * A.imag)


def refine(Fn: np.ndarray, r: float, z: float, w: float, step, half, pad: int = 16):
    """The largest power_at over the grid (r + i dr, z + j dz, w + l dw),
    |i| <= hr, |j| <= hz, |l| <= hw: returns (r, z, w, power) of the
    maximum (first in (i, j, l) order on ties) and the power at the centre."""
    dr, dz, dw = step
    hr, hz, hw = half
    best, centre = None, None
    for i in range(-hr, hr + 1):
        for j in range(-hz, hz + 1):
            for l in range(-hw, hw + 1):
                pt = (r + i * dr, z + j * dz, w + l * dw)
                P = power_at(Fn, pt[0], pt[1], pt[2], pad)
                if i == 0 and j == 0 and l == 0:
                    centre = P
                if best is None or P > best[3]:
                    best = (pt[0], pt[1], pt[2], P)
    return best, centre


def is_peak3d(Fn: np.ndarray, r: float, z: float, w: float, b: int, dz: float, dw: float, pad: int = 16) -> bool:
    """The cell (r, z, w) is not below any of its 26 neighbours
    (r +- 1/b, z +- dz, w +- dw): the 3-D local-maximum definition of a
    peak (a reading; the paper does not define its peak finder)."""
    (rr, zz, ww, P), c = refine(Fn, r, z, w, (1.0 / b, dz, dw), (1, 1, 1), pad)
    return c >= P


def search(F: np.ndarray, p: Params, bank: Bank | None = None, keep_plane: bool = False):
    """The whole path on one spectrum: normalise, plane, harmonic sums,
    statistics, max-projection, thresholds, peaks.  Candidates are sorted by
    (stage position, p)."""
    Fn = normalise(F, p.norm_block)
    P = plane(Fn, p, bank)
    res = Result()
    sums = harmonic_sums(P, p)
    for si, H in enumerate(p.stages):
        fund, S = sums[H]
        res.stats[H] = stats(S)
        th = threshold(p, si, S)
        M, arg = maxproj(fund, S)
        res.maxproj[H] = (M, arg)
        res.theta[H] = th
        for c in peaks(M, th):
            res.candidates.append((H, int(c), int(arg[c]), float(M[c])))
    res.sums = sums
    if keep_plane:
        res.plane = P
        res.normalised = Fn
    return res


# ---------------------------------------------------------------------------
# The FFT route: the whole search of a long spectrum, one row at a time
# ---------------------------------------------------------------------------

def dft(x, sign: int) -> np.ndarray:
    """X_k = sum_j x_j exp(sign 2 pi i j k / n) by the oracle's radix-2 DFT
    (n a power of two, unnormalised)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).copy()
    if _load().oracle_dft(_dp(a.view(np.float64)), a.size, int(sign)) != 0:
        raise ValueError("length must be a power of two")
    return a


def harmonic_table(p: Params):
    """harm[t, h-1] = template index of (h z_t, h w_t) for h = 1..8 (-1 off
    the grid); top[t] = number of stages at which t is a valid fundamental
    (|H z_t| <= zmax and |H w_t| <= wmax; the sets are nested in H)."""
    zt, wt = grid(p)
    T = zt.size
    harm = np.full((T, 8), -1, dtype=np.int64)
    top = np.zeros(T, dtype=np.int32)
    for t in range(T):
        z, w = int(zt[t]), int(wt[t])
        for h in range(1, 9):
            hz, hw = h * z, h * w
            if abs(hz) <= p.zmax and abs(hw) <= p.wmax:
                harm[t, h - 1] = ((hw + p.wmax) // p.dw) * p.nz + (hz + p.zmax) // p.dz
        top[t] = sum(1 for H in p.stages if abs(H * z) <= p.zmax and abs(H * w) <= p.wmax)
    return harm, top


def fft_rows(Fn: np.ndarray, p: Params, bank: Bank, templates, L: int = 8192) -> np.ndarray:
    """Power rows P[t][p], p < b N, of the given templates by the FFT route
    alone (overlap-and-save with the oracle's radix-2 DFT of length L)."""
    Fn = np.ascontiguousarray(np.asarray(Fn, dtype=np.complex128))
    tl = np.ascontiguousarray(np.asarray(templates, dtype=np.int64))
    bN = p.numbetween * Fn.size
    out = np.empty((tl.size, bN), dtype=np.float64)
    rc = _load().oracle_fft_rows(_dp(Fn.view(np.float64)), Fn.size, p.numbetween,
                                 _dp(bank.flat.view(np.float64)), _lp(bank.off), _lp(bank.D),
                                 p.n_templates, int(L), _lp(tl), tl.size, _dp(out))
    if rc != 0:
        raise ValueError("oracle_fft_rows: bad sizes")
    return out


@dataclass
class FftResult:
    candidates: list = field(default_factory=list)   # (stage, p, t, power32)
    maxproj: dict = field(default_factory=dict)      # H -> (M float32, argmax t)
    runner_up: dict = field(default_factory=dict)    # H -> second-best FP32 value per cell
    theta: dict = field(default_factory=dict)        # H -> float32
    stats: dict = field(default_factory=dict)        # H -> (mu, sd)
    sums: dict = field(default_factory=dict)         # H -> (sum S_H, sum S_H^2, cells counted)
    rows: int = 0                                    # power rows computed


def fft_search(Fn: np.ndarray, p: Params, bank: Bank | None = None, L: int = 8192,
               fund=None) -> FftResult:
    """Steps 3-7 of ``search`` for the normalised spectrum Fn by the FFT route.

    Every power row P(., z_t, w_t) is computed by overlap-and-save with the
    oracle's radix-2 FP64 DFT of length L; rows of the harmonics (h z, h w) of
    a fundamental are computed when that fundamental is processed, so the
    plane is never held.  With ``fund`` (ascending template indices) only
    those fundamentals are processed (for timing; the statistics and
    candidates then describe that subset).  Statistics: mu = E[S_H],
    sd = (E[S_H^2] - mu^2)^(1/2) over the defined cells (population values,
    FP64 sums)."""
    Fn = np.ascontiguousarray(np.asarray(Fn, dtype=np.complex128))
    harm, top = harmonic_table(p)
    T = p.n_templates
    if fund is None:
        fund = np.arange(T, dtype=np.int64)
    fund = np.ascontiguousarray(np.asarray(fund, dtype=np.int64))
    if bank is None:
        need = sorted({int(harm[t, h - 1]) for t in fund.tolist()
                       for h in range(1, p.stages[top[t] - 1] + 1)})
        bank = Bank(p, templates=need)
    bN = p.numbetween * Fn.size
    nv = [n_valid(bN, H) for H in p.stages]
    moff = np.concatenate([[0], np.cumsum(nv)[:-1]]).astype(np.int64)
    tot = int(sum(nv))
    Mv = np.full(tot, -np.inf, dtype=np.float32)
    M2 = np.full(tot, -np.inf, dtype=np.float32)
    Mt = np.full(tot, -1, dtype=np.int32)
    sums = np.zeros(2 * len(p.stages), dtype=np.float64)
    st = np.ascontiguousarray(np.array(p.stages, dtype=np.int32))
    rows = ctypes.c_int64(0)
    ip = ctypes.POINTER(ctypes.c_int32)
    fp = ctypes.POINTER(ctypes.c_float)
    rc = _load().oracle_fft_search(
        _dp(Fn.view(np.float64)), Fn.size, p.numbetween, _dp(bank.flat.view(np.float64)), _lp(bank.off),
        _lp(bank.D), T, int(L), len(p.stages), st.ctypes.data_as(ip), _lp(np.ascontiguousarray(harm)),
        top.ctypes.data_as(ip), _lp(fund), fund.size, _lp(moff), Mv.ctypes.data_as(fp),
        Mt.ctypes.data_as(ip), M2.ctypes.data_as(fp), _dp(sums), ctypes.byref(rows))
    if rc != 0:
        raise ValueError("oracle_fft_search: bad sizes (L must be a power of two above the taps)")
    res = FftResult(rows=int(rows.value))
    for si, H in enumerate(p.stages):
        a, n = int(moff[si]), nv[si]
        M, arg, sec = Mv[a:a + n].copy(), Mt[a:a + n].astype(np.int64), M2[a:a + n].copy()
        count = float(n) * float(sum(1 for t in fund.tolist() if top[t] > si))
        res.sums[H] = (float(sums[2 * si]), float(sums[2 * si + 1]), count)
        mu = sums[2 * si] / count if count > 0 else 0.0
        sd = math.sqrt(max(0.0, sums[2 * si + 1] / count - mu * mu)) if count > 0 else 0.0
        res.stats[H] = (mu, sd)
        th = np.float32(p.thresh[si]) if p.thresh_mode == "abs" else np.float32(mu + p.thresh[si] * sd)
        res.theta[H] = th
        res.maxproj[H] = (M, arg)
        res.runner_up[H] = sec
        for c in peaks(M, th):
            res.candidates.append((H, int(c), int(arg[c]), float(M[c])))
    return res


# ---------------------------------------------------------------------------
# The harmonic sum indexed by the highest harmonic (sub-harmonic form)
# ---------------------------------------------------------------------------

def round_ratio(a, h: int, H: int):
    """Nearest integer to a h / H, halves rounded away from zero (integer
    arithmetic; a may be an array of any sign)."""
    a = np.asarray(a, dtype=np.int64)
    m = np.abs(a) * h
    q = (2 * m + H) // (2 * H)
    return np.sign(a) * q


def subharmonic_templates(p: Params, H: int) -> np.ndarray:
    """sub[t, h-1] = template index of (z_h, w_h), the grid point nearest to
    (h z_t / H, h w_t / H) for h = 1..H (reading: the sub-harmonic terms of a
    top harmonic at (z_t, w_t), rounded on the grid, halves away from zero)."""
    zt, wt = grid(p)
    zi = zt // p.dz
    wi = wt // p.dw
    sub = np.empty((zt.size, H), dtype=np.int64)
    for h in range(1, H + 1):
        zh = round_ratio(zi, h, H)
        wh = round_ratio(wi, h, H)
        sub[:, h - 1] = (wh + p.wmax // p.dw) * p.nz + (zh + p.zmax // p.dz)
    return sub


def subharmonic_sums(P: np.ndarray, p: Params, H: int) -> np.ndarray:
    """S'_H[t, q] = sum_{h=1..H} P[t_h, round(h q / H)] for every template t
    (the top harmonic) and every cell q < b N, FP64 in h order: the harmonic
    sum of a signal whose H-th harmonic sits at (q, z_t, w_t) (the form of
    Ransom's harmonic summing that the paper's method lineage uses, Sec. 3
    names the harmonic sum; the rounding is a reading)."""
    sub = subharmonic_templates(p, H)
    q = np.arange(P.shape[1], dtype=np.int64)
    S = np.zeros(P.shape, dtype=np.float64)
    for h in range(1, H + 1):
        S += P[sub[:, h - 1]][:, round_ratio(q, h, H)]
    return S


def subharmonic_search(F: np.ndarray, p: Params, bank: Bank | None = None):
    """The whole path with the sub-harmonic form of every stage: plane,
    S'_H over all templates and cells, statistics, max-projection over
    (z, w) (FP32 decisions, lowest t on ties), thresholds and peaks.
    Returns a Result (sums[H] = (all templates, S'_H))."""
    Fn = normalise(F, p.norm_block)
    P = plane(Fn, p, bank)
    res = Result()
    allt = np.arange(p.n_templates, dtype=np.int64)
    for si, H in enumerate(p.stages):
        S = P if H == 1 else subharmonic_sums(P, p, H)
        res.stats[H] = stats(S)
        th = threshold(p, si, S)
        M, arg = maxproj(allt, S)
        res.maxproj[H] = (M, arg)
        res.theta[H] = th
        res.sums[H] = (allt, S)
        for c in peaks(M, th):
            res.candidates.append((H, int(c), int(arg[c]), float(M[c])))
    return res
