"""Writes the FP64 oracle's result for the paper-scale search (the benchmark's
workload) under tests/golden/.

Calls only ``oracle`` and ``synth`` (never the CUDA path).  The search runs by
the oracle's FFT route (``oracle.fft_search``: overlap-and-save with its own
radix-2 FP64 DFT, one power row at a time), because direct summation over
2^23 cells x 12 261 templates is out of reach on a CPU.  About 15 minutes
on 8 cores.  Run from the repository root:

    python tests/golden/make_paper_scale.py

Workload: ``synth.paper_scale()`` -- 2^22 bins, noise plus 8 chirps; zmax 200
(dz 2), wmax 600 (dw 20): 12 261 templates; harmonic stages 1, 2, 4, 8;
thresholds theta_H = mu_H + T_H sigma_H with T = 19, 17, 15, 14 (the paper's
mean / standard-deviation candidate selection, Sec. 3).

Files:
  paper_scale_candidates.json  per stage: mu, sigma, theta, cells, the
      candidates (p, t, M, runner-up, M(p-1), M(p+1)) and the cells that are
      near a candidate decision without being one (same fields), within
      NEAR_REL x H x (the plane maximum) of the threshold or of a neighbour;
  paper_scale_maxproj_sample.npz  per stage H: cells ``p<H>`` (65 536 drawn
      at random plus +-4 around every candidate), with M_H ``m<H>``, its
      argmax ``t<H>`` and the runner-up ``s<H>`` at those cells.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402

T_SIGMA = (19.0, 17.0, 15.0, 14.0)
FFT_LEN = 8192
NEAR_REL = 2e-3        # 20 x the 1e-4 parity tolerance
SAMPLE = 65536


def main():
    t0 = time.time()
    wl = synth.paper_scale()
    p = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=wl.stages, thresh_mode="sigma", thresh=T_SIGMA)
    F = wl.make()
    Fn = oracle.normalise(F, p.norm_block)
    bank = oracle.Bank(p)
    t1 = time.time()
    res = oracle.fft_search(Fn, p, bank=bank, L=FFT_LEN)
    t2 = time.time()
    plane_max = float(res.maxproj[1][0].max())
    out = {"workload": wl.name, "oracle": "FP64 FFT route (oracle.fft_search), L = %d" % FFT_LEN,
           "params": {"zmax": p.zmax, "dz": p.dz, "wmax": p.wmax, "dw": p.dw, "numbetween": p.numbetween,
                      "pad_bins": p.pad_bins, "stages": list(p.stages), "thresh_mode": p.thresh_mode,
                      "thresh": list(p.thresh), "norm_block": p.norm_block},
           "plane_max": plane_max, "near_rel": NEAR_REL, "rows": res.rows,
           "seconds": {"taps": round(t1 - t0, 1), "search": round(t2 - t1, 1), "threads": oracle.threads()},
           "stages": {}}
    arrays = {}
    for H in p.stages:
        M, arg = res.maxproj[H]
        sec = res.runner_up[H]
        th = float(res.theta[H])
        mu, sd = res.stats[H]
        n = M.size
        m64 = M.astype(np.float64)
        left = np.concatenate([[-np.inf], m64[:-1]])
        right = np.concatenate([m64[1:], [-np.inf]])
        cand = set(int(c[1]) for c in res.candidates if c[0] == H)
        g = NEAR_REL * H * plane_max
        near = np.nonzero((m64 > th - g) & (m64 > left - g) & (m64 >= right - g))[0]

        def rec(q):
            return [int(q), int(arg[q]), float(M[q]), float(sec[q]),
                    float(left[q]) if q > 0 else None, float(right[q]) if q + 1 < n else None]

        out["stages"][str(H)] = {
            "mu": mu, "sigma": sd, "theta": th, "cells": n,
            "candidates": [rec(q) for q in sorted(cand)],
            "near": [rec(int(q)) for q in near if int(q) not in cand]}
        rng = np.random.default_rng(7000 + H)
        ps = set(rng.choice(n, SAMPLE, replace=False).tolist())
        for q in cand:
            ps.update(range(max(0, q - 4), min(n, q + 5)))
        ps = np.array(sorted(ps), dtype=np.int64)
        arrays["p%d" % H] = ps.astype(np.int32)
        arrays["m%d" % H] = M[ps]
        arrays["t%d" % H] = arg[ps].astype(np.int32)
        arrays["s%d" % H] = sec[ps]
    with open(os.path.join(HERE, "paper_scale_candidates.json"), "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")
    np.savez_compressed(os.path.join(HERE, "paper_scale_maxproj_sample.npz"), **arrays)
    print("taps %.0f s, search %.0f s, %d rows, %d candidates" % (t1 - t0, t2 - t1, res.rows,
                                                                   len(res.candidates)))


if __name__ == "__main__":
    main()
