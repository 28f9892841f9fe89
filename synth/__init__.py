"""Seeded synthetic inputs for the Fourier-domain jerk search.

This module is shared by the FP64 oracle (``oracle/``), the tests and the
benchmark.  It holds none of the search's own arithmetic (no response
function, no templates, no correlation): it only *simulates data*, i.e. a
complex time series made of white noise plus pulsar-like chirps, and takes
its discrete Fourier transform with a library FFT.

Conventions (the paper defines z = fdot T^2 and w = fddot T^3, Sec. 2):

* A signal is ``amp * exp(i (phase + 2 pi (r u + z u^2/2 + w u^3/6)))`` with
  ``u = t/T - 1/2`` the time measured from the middle of the observation, so
  that (r, z, w) are the Fourier frequency, its first and its second
  derivative at mid-observation.
* Sample n sits at the middle of its interval, ``u_n = (n + 1/2)/N - 1/2``,
  and the spectrum is taken with the same time origin:
  ``F_k = (1/N) sum_n x_n exp(-2 pi i k u_n)``, which is
  ``(-1)^k exp(-i pi k / N) fft(x)[k] / N``.
* Noise is drawn directly in the Fourier domain, ``F_k = (x + i y)/sqrt(2)``
  with x, y ~ N(0, 1), so that E|F_k|^2 = 1 and a signal of amplitude
  ``sqrt(S)`` has power S against unit-mean noise.

Every generator takes an explicit seed (NumPy PCG64) and returns complex64
arrays (generated in FP64 and rounded once).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Signal:
    """One injected chirp: mid-observation (r, z, w), power SNR, phase."""
    r: float
    z: float
    w: float
    snr: float
    phase: float = 0.0


def noise(n: int, seed: int) -> np.ndarray:
    """Unit-power complex Gaussian noise, complex128[n]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    return (x + 1j * y) / math.sqrt(2.0)


def chirp_spectrum(n: int, signals, harmonics: int = 1) -> np.ndarray:
    """Spectrum (complex128[n]) of a sum of chirps sampled at n points.

    With ``harmonics = H`` every signal also gets harmonics h = 2..H at
    (h r, h z, h w) with the same power ``snr`` each and phase ``h * phase``.
    """
    u = (np.arange(n, dtype=np.float64) + 0.5) / n - 0.5
    x = np.zeros(n, dtype=np.complex128)
    for s in signals:
        amp = math.sqrt(s.snr)
        for h in range(1, harmonics + 1):
            cyc = (h * s.r) * u + (h * s.z) * u * u / 2.0 + (h * s.w) * u ** 3 / 6.0
            cyc = cyc - np.floor(cyc)          # keep the phase argument small
            x += amp * np.exp(1j * (h * s.phase + 2.0 * math.pi * cyc))
    k = np.arange(n)
    spec = np.fft.fft(x) / n
    # time origin at mid-observation: (-1)^k exp(-i pi k / n)
    shift = np.where(k % 2 == 0, 1.0, -1.0) * np.exp(-1j * np.pi * k / n)
    return spec * shift


def spectrum(n: int, seed: int, signals=(), harmonics: int = 1,
             with_noise: bool = True) -> np.ndarray:
    """Noise (seeded) plus injected signals, rounded to complex64[n]."""
    f = noise(n, seed) if with_noise else np.zeros(n, dtype=np.complex128)
    if signals:
        f = f + chirp_spectrum(n, signals, harmonics)
    return f.astype(np.complex64)


# --------------------------------------------------------------------------
# Search configurations.  Each names the workload by what it is.
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n_bins: int
    zmax: int
    dz: int
    wmax: int
    dw: int
    stages: tuple
    thresh: tuple            # ABS thresholds (normalised power units) per stage
    seed: int
    signals: list = field(default_factory=list)
    harmonics: int = 1

    def make(self) -> np.ndarray:
        return spectrum(self.n_bins, self.seed, self.signals, self.harmonics)

    @property
    def n_templates(self) -> int:
        return (2 * self.zmax // self.dz + 1) * (2 * self.wmax // self.dw + 1)

    @property
    def cells(self) -> int:
        return 2 * self.n_bins * self.n_templates


def small_single() -> Workload:
    """2^16 bins, one chirp at (10000.25, 12, 40) with power SNR 30;
    z in [-20, 20] step 2, w in [-60, 60] step 20 (147 templates);
    harmonic stages {1, 2}."""
    rng = np.random.Generator(np.random.PCG64(1001))
    sig = Signal(10000.25, 12.0, 40.0, 30.0, float(rng.uniform(0, 2 * math.pi)))
    return Workload("spectrum 2^16 bins, zmax 20, wmax 60, 147 templates, stages 1-2",
                    1 << 16, 20, 2, 60, 20, (1, 2), (15.0, 20.0), 1, [sig])


def paper_scale(n: int = 1 << 22) -> Workload:
    """2^22 bins (or n), 8 chirps with r, z in [-200, 200], w in [-600, 600]
    drawn uniformly (SNR uniform in [20, 50]); z in [-200, 200] step 2, w in
    [-600, 600] step 20 (12 261 templates); harmonic stages {1, 2, 4, 8}."""
    rng = np.random.Generator(np.random.PCG64(2002))
    sigs = []
    for _ in range(8):
        sigs.append(Signal(float(rng.uniform(1024, n - 1024)),
                           float(rng.uniform(-200, 200)),
                           float(rng.uniform(-600, 600)),
                           float(rng.uniform(20, 50)),
                           float(rng.uniform(0, 2 * math.pi))))
    return Workload("spectrum 2^%d bins, zmax 200, wmax 600, 12261 templates, stages 1-2-4-8"
                    % int(round(math.log2(n))),
                    n, 200, 2, 600, 20, (1, 2, 4, 8), (20.0, 26.0, 34.0, 48.0), 2, sigs)


def dm_trials(count: int = 64, seed: int = 3, lo: float = 20.0, hi: float = 22.0):
    """``count`` spectra of uneven length floor(2^U(lo, hi)) bins, each with
    0-3 chirps (z in [-200, 200], w in [-300, 300]).  Returns a list of
    (n_bins, seed, signals)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(math.floor(2.0 ** rng.uniform(lo, hi)))
        ns = int(rng.integers(0, 4))
        sigs = [Signal(float(rng.uniform(1024, n - 1024)), float(rng.uniform(-200, 200)),
                       float(rng.uniform(-300, 300)), float(rng.uniform(20, 50)),
                       float(rng.uniform(0, 2 * math.pi))) for _ in range(ns)]
        out.append((n, seed * 1000 + i, sigs))
    return out
