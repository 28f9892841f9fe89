#!/usr/bin/env python
"""Benchmark of the GB300 Fourier-domain jerk search.

Metric: template-bins/s (f-fdot-fddot cells per second) = b N nz nw / time of
one search step (jerk_search + jerk_candidates), whole job over all ranks.

Workload (default): one 2^22-bin complex FP32 spectrum, unit noise plus 8
injected chirps; z in [-200, 200] step 2, w in [-600, 600] step 20 (12 261
templates); interbinning (2 cells per bin); harmonic stages {1, 2, 4, 8};
thresholds mu + T sigma (SIGMA mode, the paper's mean/standard deviation
candidate selection).  Inputs are synthetic (``synth``).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank searches its own spectrum (independent DM trials:
weak scaling, no collective on the data path).  ``--impl reference`` times
the FP64 CPU oracle on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "template-bins/sec (f-fdot-fddot cells/s)"
UNIT = "cells/s"
SIGMA_T = (19.0, 17.0, 15.0, 14.0)
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_DEFAULT = 2070.0


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("paper", "small", "dm", "serve"), default="paper",
                    help="paper: one 2^22-bin spectrum; small: 2^16 bins; dm: 64 uneven DM-trial spectra "
                         "searched in batches (the batched form) and one by one (the per-spectrum form); "
                         "serve: Poisson arrivals served by the continuous-batching server and one by one")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: arrivals per second")
    ap.add_argument("--duration", type=float, default=20.0, help="serve: seconds of arrivals")
    ap.add_argument("--workers", type=int, default=4, help="serve: plans sharing the bank")
    ap.add_argument("--dm-count", type=int, default=64)
    ap.add_argument("--autotune", action="store_true",
                    help="pick the tile shape (segment length, template group size) by timing (cached)")
    ap.add_argument("--group-size", type=int, default=0, help="templates per template group (0: the library's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seg-len", type=int, default=0)
    ap.add_argument("--stages", default="",
                    help="harmonic stages of the paper-scale search, e.g. 1 or 1,2,4 (default: the "
                         "workload's 1,2,4,8)")
    ap.add_argument("--precision", type=int, default=0, choices=(0, 1, 2),
                    help="filter arithmetic: 0 FP32, 1 BF16 tensor-core DFT blocks, 2 FP16 tensor-core DFT blocks")
    ap.add_argument("--bins", type=int, default=1 << 22,
                    help="spectrum length of the paper-scale bank (smaller for profiling)")
    return ap.parse_args()


def workload(name, bins=1 << 22, stages=""):
    import dataclasses

    import synth
    wl = synth.paper_scale(bins) if name == "paper" else synth.small_single()
    if stages:
        st = tuple(int(x) for x in stages.split(","))
        wl = dataclasses.replace(wl, stages=st, thresh=tuple(wl.thresh[:len(st)]),
                                 name=wl.name.replace("stages 1-2-4-8", "stages " + "-".join(map(str, st))))
    return wl


def peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def conv_flops_per_cell(L, V):
    """Algorithmic FP32 flops per output cell of the fused kernel: one inverse
    FFT (5 L log2 L), the template multiply (6 L) and |.|^2 (3 V) per
    (segment, template), spread over the V cells kept."""
    return (5.0 * L * math.log2(L) + 6.0 * L + 3.0 * V) / V


def kernel_hash(main="conv.cu"):
    h = hashlib.sha256()
    for f in (main, "fft.cuh", "device_sync.cuh", "rows.cuh"):
        with open(os.path.join(ROOT, "paper_1911_01353_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


TRAFFIC_FILES = {0: "conv_kernel_traffic_2p16bins.txt", 1: "conv_tc_kernel_traffic_2p16bins.txt",
                 2: "conv_tc_kernel_traffic_2p16bins.txt"}


def conv_algorithmic_bytes(slot_floats, n_templates, L, n_bins):
    """Bytes one filter launch must move: the harmonic rows it writes, the
    template bank and the spectrum it reads, the stage-1 max-projection."""
    return 4 * slot_floats + 8 * n_templates * L + 8 * n_bins + 8 * 2 * n_bins


def recorded_traffic(L, alg_bytes, precision=0):
    """DRAM bytes (read + write) per launch of the filter kernel (FP32, or the
    tensor-core kernel for precision 1/2), from the committed ncu record of a
    small case (one launch, 2^16 bins, the full bank: a few GB on the device),
    scaled to this launch by the ratio of the two launches' algorithmic bytes
    (``conv_algorithmic_bytes``).  Returns (bytes, note), or (None, why) when
    no record was taken on the current kernel sources."""
    name = TRAFFIC_FILES[precision]
    main = "conv.cu" if precision == 0 else "conv_tc.cu"
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None, "no record"
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_sha") != kernel_hash(main) or int(vals.get("seg_len", 0)) != L:
        return None, "record taken on other kernel sources"
    if precision and int(vals.get("precision", 0)) != precision:
        return None, "record taken at another precision"
    try:
        small = float(vals["dram_bytes_per_launch"])
        small_alg = float(vals["algorithmic_bytes_per_launch"])
        bins = int(vals["bins"])
    except (KeyError, ValueError):
        return None, "malformed record"
    return small * alg_bytes / small_alg, (
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at %d bins (profiles/%s, "
        "%.3f x its algorithmic bytes), scaled by algorithmic bytes (%.4g per launch here)"
        % (bins, name, small / small_alg, alg_bytes))


def recorded_limiter(L, precision=0):
    """Pipe utilisations of the filter kernel from the committed ncu section
    capture of the same small case (one launch, 2^16 bins, the full bank), kept
    in the traffic record beside the DRAM bytes: which unit bounds the kernel.
    None when the record is missing or was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", TRAFFIC_FILES[precision])
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    main = "conv.cu" if precision == 0 else "conv_tc.cu"
    if vals.get("kernel_sha") != kernel_hash(main) or int(vals.get("seg_len", 0)) != L:
        return None
    out = {}
    for k in ("l1tex_throughput_pct", "issue_active_pct", "fma_pipe_pct", "tensor_pipe_pct"):
        if k in vals:
            out[k] = float(vals[k])
    if not out:
        return None
    out["source"] = "ncu --set full, one launch at %s bins (profiles/%s)" % (vals.get("bins"), TRAFFIC_FILES[precision])
    return out


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = tempfile.mktemp(prefix="clocks", suffix=".csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if self.bus_id:
            mine = [r for r in rows if self.bus_id.endswith(r[1].lower()[-12:]) or r[1].lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        idx0 = rows[0][0]
        rows = [r for r in rows if r[0] == idx0]
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(wl, spec, n_fund=1024):
    """Time the FP64 oracle's FFT route (``oracle.fft_search``: normalisation,
    forward DFTs of every segment, then per fundamental its own power row and
    the rows of its harmonics, with the max-projections and statistics) on
    n_fund fundamentals spread evenly over the bank.  The whole search needs
    one row per (fundamental, harmonic) pair; the sample's time is scaled up
    by rows.  Template taps are built first and not timed (plan time, like
    the GPU's template bank).  Returns (cells/s, cells, threads, description,
    seconds)."""
    import numpy as np

    import oracle
    op = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=wl.stages, thresh_mode="sigma",
                       thresh=SIGMA_T[:len(wl.stages)])
    T = op.n_templates
    harm, top = oracle.harmonic_table(op)
    rows_full = int(sum(op.stages[int(top[t]) - 1] for t in range(T)))
    fund = np.unique(np.linspace(0, T - 1, min(n_fund, T)).astype(np.int64))
    need = sorted({int(harm[t, h - 1]) for t in fund.tolist() for h in range(1, op.stages[int(top[t]) - 1] + 1)})
    bank = oracle.Bank(op, templates=need)                      # taps: not timed
    t0 = time.perf_counter()
    Fn = oracle.normalise(spec, op.norm_block)
    res = oracle.fft_search(Fn, op, bank=bank, fund=fund)
    dt = time.perf_counter() - t0
    cells_full = 2 * wl.n_bins * T
    cells = cells_full * res.rows / rows_full                   # the sample's share of the search
    desc = ("FP64 FFT route of the oracle (overlap-and-save, radix-2 DFT of length 8192) for %d of %d "
            "fundamentals (evenly spaced): %d of the search's %d power rows, with harmonic sums, "
            "max-projections and statistics, over the whole %d-bin spectrum; normalisation and segment "
            "DFTs timed, template taps not; scaled to the whole search by rows"
            % (fund.size, T, res.rows, rows_full, wl.n_bins))
    return cells / dt, cells, oracle.threads(), desc, dt


def tc_accuracy(wl, spec, plan, x, fp32_cands, tc_cands, cells=65536):
    """Error of the reduced-precision filter against the FP64 oracle on a
    sample: three runs of 64 consecutive templates (z from -128 to -2 + 126 at
    w = -wmax, 0, +wmax) over `cells` cells in the middle of the spectrum
    (the plane rows come from jerk_plane, the reference from the oracle's
    direct correlation).  Also the candidate agreement with the FP32 filter on
    the whole workload."""
    import numpy as np
    import torch

    import oracle
    op = oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=wl.stages)
    zt, wt = oracle.grid(op)
    nz, nw = 2 * wl.zmax // wl.dz + 1, 2 * wl.wmax // wl.dw + 1
    p0 = wl.n_bins - cells // 2
    Fn = oracle.normalise(spec, op.norm_block)
    i0 = max(0, nz // 2 - 64)
    errs, refmax, sq, cnt = [], 0.0, 0.0, 0
    for j in (0, nw // 2, nw - 1):
        t0 = j * nz + i0
        nt = min(64, nz - i0)
        out = torch.empty((nt, 2 * wl.n_bins), dtype=torch.float32, device=x.device)
        plan.plane(x, t0, nt, out)
        got = out[:, p0:p0 + cells].cpu().numpy().astype(np.float64)
        for k in range(nt):
            t = t0 + k
            c = oracle.taps(int(zt[t]), int(wt[t]), op.numbetween, op.pad_bins)
            o = oracle.correlate(Fn, c, op.numbetween, p0, cells)
            ref = o.real * o.real + o.imag * o.imag
            d = np.abs(got[k] - ref)
            errs.append(float(d.max()))
            sq += float((d * d).sum())
            cnt += d.size
            refmax = max(refmax, float(ref.max()))
    a, b = set(fp32_cands), set(tc_cands)
    return {"vs": "FP64 oracle, direct correlation", "templates": 3 * 64, "cells": cells,
            "max_err_rel_plane_max": max(errs) / refmax, "rms_err_rel_plane_max": (sq / cnt) ** 0.5 / refmax,
            "candidates_fp32": len(a), "candidates": len(b), "common": len(a & b),
            "only_fp32": len(a - b), "only_this": len(b - a)}


def reference_arm(a):
    """The oracle (there is no reference code: the reference is a paper) on
    this arm's workload and metric: each step times its FFT route on a bounded
    sample of fundamentals, sized so that the whole run takes about two
    minutes."""
    wl = workload(a.workload, a.bins, a.stages)
    spec = wl.make()
    steps = a.warmup + a.steps
    # calibrate: rows per second of this host on a small sample
    v, n, th, desc, dt = oracle_sample(wl, spec, n_fund=8)
    per_step = max(1.0, 120.0 / max(1, steps))
    n_fund = int(max(2, min(512, 8 * per_step / max(dt, 1e-3))))
    times, cells = [], 0.0
    for i in range(steps):
        v, n, th, desc, dt = oracle_sample(wl, spec, n_fund=n_fund)
        if i >= a.warmup:
            times.append(dt)
            cells += n
    value = cells / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(times) / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle FFT route", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def dm_bench(a):
    """64 DM-trial spectra of lengths 2^U(20,22) (zmax 200, wmax 300, stages
    1-2-4-8, SIGMA thresholds): the batched form (jerk_search_batch with graph
    replay, spectra packed into batches of at most 2^23 bins) against the
    per-spectrum form (jerk_search on each), same plan, same candidates."""
    import numpy as np
    import torch

    import paper_1911_01353_gb300 as pkg
    import synth
    from paper_1911_01353_gb300 import autotune
    from paper_1911_01353_gb300 import build as pkg_build
    pkg_build.build()
    torch.cuda.set_device(0)
    trials = synth.dm_trials(a.dm_count, seed=3)
    specs = [synth.spectrum(n, seed, sigs) for n, seed, sigs in trials]
    zmax, dz, wmax, dw, stages = 200, 2, 300, 20, (1, 2, 4, 8)
    max_bins = 1 << 23
    seg_len, group_size = (autotune.best_shape(zmax, dz, wmax, dw, stages, 1 << 21) if a.autotune
                           else (a.seg_len, a.group_size))
    p = pkg.make_params(zmax, dz, wmax, dw, stages=stages, thresh=SIGMA_T, thresh_mode=pkg.THRESH_SIGMA,
                        seg_len=seg_len, max_bins=max_bins, max_candidates=1 << 22, max_batch=16,
                        group_size=group_size)
    plan = pkg.Plan(p)
    dev = [torch.from_numpy(s).cuda() for s in specs]
    batches, cur, tot = [], [], 0
    for i, s in enumerate(specs):
        if cur and (tot + s.size > max_bins or len(cur) == 16):
            batches.append(cur)
            cur, tot = [], 0
        cur.append(i)
        tot += s.size
    batches.append(cur)
    cells = sum(2 * s.size for s in specs) * plan.info.n_templates
    stream = torch.cuda.current_stream()

    def batched():
        out = []
        for bt in batches:
            plan.search_batch([dev[i] for i in bt], graph=True)
            out += [(bt[c.item], c.stage, c.p, c.t, c.power) for c in plan.candidates()]
        return out

    def single():
        out = []
        for i in range(len(specs)):
            plan.search(dev[i])
            out += [(i, c.stage, c.p, c.t, c.power) for c in plan.candidates()]
        return out

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        res = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), res

    for _ in range(max(1, a.warmup)):
        batched()
        single()
    tb_ms, tsingle_ms = [], []
    rb = rs = None
    for _ in range(a.steps):
        t, rb = timed(batched)
        tb_ms.append(t)
        t, rs = timed(single)
        tsingle_ms.append(t)
    same = sorted(rb) == sorted(rs)
    vb = cells / (statistics.median(tb_ms) / 1e3)
    vs = cells / (statistics.median(tsingle_ms) / 1e3)
    line = {"metric": METRIC, "value": vb, "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": statistics.median(tb_ms), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%d DM-trial spectra of 2^U(20,22) bins, zmax 200, wmax 300, %d templates, "
                                   "stages 1-2-4-8" % (len(specs), plan.info.n_templates),
                       "total_bins": int(sum(s.size for s in specs)), "batches": len(batches),
                       "seg_len": plan.info.seg_len, "graph": True},
            "per_spectrum_form": {"value": vs, "unit": UNIT, "ms": statistics.median(tsingle_ms)},
            "batched_over_per_spectrum": vb / vs,
            "candidates": len(rb), "identical_candidates": same}
    print(json.dumps(line))
    plan.close()


def serve_bench(a):
    """Serving: Poisson arrivals (a.rate per second for a.duration s, seed 5)
    of requests with lengths log-uniform in 2^18..2^23 bins, zmax in {50, 100,
    200, 300}, wmax in {0, 300, 600, 900}; one bank for (300, 900) resident on
    the device, stage 1 (matched filter + candidate selection, SIGMA T = 19).
    The same trace runs through the continuous-batching server and through
    the plain form (one request at a time, first come first served); both
    report template-bins/s over the run and p50/p99 latency from arrival."""
    import numpy as np
    import torch

    import synth
    from paper_1911_01353_gb300 import build as pkg_build
    from paper_1911_01353_gb300 import jerk, serve
    pkg_build.build()
    torch.cuda.set_device(0)
    dz, dw = 2, 20
    trace = serve.poisson_trace(a.rate, a.duration, seed=5)
    warm = serve.poisson_trace(a.rate, 1.0, seed=6)
    # four base spectra of 2^23 bins (noise + 6 chirps each); a request of n
    # bins is the first n bins of one of them, from pinned host memory
    rng = np.random.default_rng(5)
    base = []
    for k in range(4):
        n = 1 << 23
        sigs = [synth.Signal(float(rng.uniform(600, (1 << 18) - 600)) if i < 3 else float(rng.uniform(600, n - 600)),
                             float(rng.uniform(-300, 300)), float(rng.uniform(-900, 900)),
                             float(rng.uniform(30, 60)), float(rng.uniform(0, 6.28)))
                for i in range(6)]
        base.append(torch.from_numpy(synth.spectrum(n, 50 + k, sigs)).pin_memory())

    def requests(tr, rid0=0):
        return [serve.Request(rid0 + i, base[(rid0 + i) % 4][:n], zs, ws, arrival=t)
                for i, (t, n, zs, ws) in enumerate(tr)]

    t0 = time.perf_counter()
    srv = serve.Server(300, 900, dz=dz, dw=dw, stages=(1,), thresh=(19.0,), thresh_mode=jerk.THRESH_SIGMA,
                       n_workers=a.workers, worker_bins=1 << 24, max_batch=32, max_candidates=1 << 22,
                       precision=a.precision)
    bank_s = time.perf_counter() - t0
    bus = getattr(torch.cuda.get_device_properties(0), "pci_bus_id", None)
    clk = ClockSampler(str(bus) if bus is not None else None)
    out = {}
    for name, kw in (("served", dict()), ("plain", dict(n_workers=1, max_batch=1, fifo=True))):
        srv.run(requests(warm, 100000), **kw)                     # warm-up
        if name == "served":
            clk.start()
        done = srv.run(requests(trace), **kw)
        if name == "served":
            clocks = clk.stop()
        out[name] = (serve.summary(done, dz, dw), {r.rid: r.candidates for r in done})
    same = out["served"][1] == out["plain"][1]
    sv, pl = out["served"][0], out["plain"][0]
    line = {"metric": METRIC + "; p50/p99 latency", "value": sv["cells_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": sv["seconds"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": ("f32", "bf16", "f16")[a.precision],
            "data": "synthetic",
            "config": {"workload": "serving: Poisson %.0f req/s for %.0f s, n = 2^U(18,23) bins, zmax in "
                                   "{50,100,200,300}, wmax in {0,300,600,900}, one (300, 900) bank of %d "
                                   "templates, stage 1" % (a.rate, a.duration, srv.bank.info.n_templates),
                       "requests": sv["requests"], "workers": a.workers, "seg_len": srv.bank.info.seg_len,
                       "bank_bytes": srv.bank.info.bank_bytes, "bank_build_s": bank_s},
            "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"], "mean_ms": sv["mean_ms"],
            "plain_form": {"value": pl["cells_per_s"], "p50_ms": pl["p50_ms"], "p99_ms": pl["p99_ms"],
                           "seconds": pl["seconds"]},
            "served_over_plain": sv["cells_per_s"] / pl["cells_per_s"],
            "offered_cells_per_s": sv["cells"] / a.duration,
            "identical_candidates": same, "clocks": clocks}
    print(json.dumps(line))
    srv.close()


def main():
    a = args_()
    if a.workload == "serve" and a.impl == "ours":
        return serve_bench(a)
    if a.workload == "dm" and a.impl == "ours":
        dm_bench(a)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        if rank == 0:
            reference_arm(a)
        return

    import numpy as np
    import torch

    import paper_1911_01353_gb300 as pkg
    from paper_1911_01353_gb300 import build as pkg_build
    pkg_build.build()

    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)

    import synth
    wl = workload(a.workload, a.bins, a.stages)
    spec = synth.spectrum(wl.n_bins, wl.seed + 1000 * rank, wl.signals) if rank else wl.make()
    seg_len, group_size = a.seg_len, a.group_size
    if a.autotune and world == 1:
        from paper_1911_01353_gb300 import autotune
        seg_len, group_size = autotune.best_shape(wl.zmax, wl.dz, wl.wmax, wl.dw, wl.stages, wl.n_bins,
                                                  device=local)
    p = pkg.make_params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=wl.stages,
                        thresh=SIGMA_T[:len(wl.stages)], thresh_mode=pkg.THRESH_SIGMA,
                        seg_len=seg_len, max_bins=wl.n_bins, max_candidates=1 << 20, precision=a.precision,
                        group_size=group_size)
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    plan = pkg.Plan(p, device=local, stream=stream)
    stream.synchronize()
    t_templates = time.perf_counter() - t0
    L, V = plan.info.seg_len, plan.info.seg_valid
    cells = 2 * wl.n_bins * plan.info.n_templates

    d_spec = torch.from_numpy(spec).cuda()
    h_spec = torch.from_numpy(spec).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    plan.profile(True)

    def step(host=False):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if host:
            plan.search_host(h_spec.numpy(), stream=stream)
        else:
            plan.search(d_spec, stream=stream)
        c = plan.candidates()
        e1.record(stream)
        return e0, e1, c

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    # FP32 FMA rate and L2 read bandwidth of this GPU (microbenchmarks, outside the timed region)
    f32, l2 = pkg.measure_peaks(local)
    f32x2 = pkg.measure_packed_fma(local)
    measured_peaks = {"fp32_fma_tflops": f32, "fp32_packed_fma_tflops": f32x2, "l2_read_gbs": l2,
                      "note": "microbenchmarks: independent FMA chains on every SM, scalar and packed (f32x2); "
                              "64 MB read 20x from L2"}

    props = torch.cuda.get_device_properties(local)
    bus = None
    for attr in ("pci_bus_id",):
        bus = getattr(props, attr, None)
    clocks = ClockSampler(str(bus) if bus is not None else None)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs, phases = [], []
    ncand = 0
    for _ in range(a.steps):
        e0, e1, c = step()
        evs.append((e0, e1))
        phases.append(plan.phase_times())
        ncand = len(c)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    # end to end: host spectrum in, candidates out, through the C ABI
    e2e_ms = []
    for _ in range(a.steps):
        e0, e1, c = step(host=True)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()

    from paper_1911_01353_gb300.ranks import max_over_ranks
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    e2e_total = max_over_ranks(sum(e2e_ms), dist, "cuda")

    value = world * cells * a.steps / (total_ms / 1e3)
    e2e_value = world * cells * a.steps / (e2e_total / 1e3)
    conv_ms = statistics.mean(ph["conv"] for ph in phases)
    flops = conv_flops_per_cell(L, V) * cells
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max_mhz = float(peaks_file()[0].get("sm_max_mhz") or SM_MAX_MHZ_DEFAULT)
    peak_alu = sms * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12    # TFLOP/s, FP32 FMA
    achieved = flops / (conv_ms / 1e3) / 1e12
    alg_bytes = conv_algorithmic_bytes(plan.info.slot_floats, plan.info.n_templates, L, wl.n_bins)
    traffic, traffic_note = recorded_traffic(L, alg_bytes, a.precision)
    peaks, peaks_src = peaks_file()

    roof = {"bound": "alu", "kernel": "conv_kernel (fused FFT-multiply-IFFT-power)",
            "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
            "frac": achieved / peak_alu, "traffic": traffic, "traffic_note": traffic_note,
            "limiter": recorded_limiter(L, 0),
            "algorithmic_bytes": alg_bytes,
            "flops_per_cell": conv_flops_per_cell(L, V),
            "peak_source": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (derived)" % (sms, sm_max_mhz),
            "measured": measured_peaks}
    # the second kernel of the step, bound by HBM: every harmonic row is read once
    # (the plan's row workspace, sized for this spectrum) and M_H written once
    harm_roof = None
    harm_ms = statistics.mean(ph["harmonic"] for ph in phases)
    if harm_ms > 0 and len(wl.stages) > 1:
        bN = 2 * wl.n_bins
        h_bytes = 4 * plan.info.slot_floats + 8 * sum((bN - 1) // H + 1 for H in wl.stages[1:])
        h_gbs = h_bytes / (harm_ms / 1e3) / 1e9
        harm_roof = {"bound": "hbm", "kernel": "harmonic_kernel (stages > 1)", "achieved": h_gbs,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": h_gbs / peaks["hbm_gbs"],
                     "bytes_per_launch": h_bytes,
                     "peak_source": "%s copy bandwidth" % peaks_src}
    accuracy = None
    if a.precision:
        # tensor pipe: two 64-point DFT blocks per point and transform, 8 flops per
        # point per unit of radix (complex products as real block products)
        tflops_cell = 8.0 * (64 + 64) * L / V
        t_achieved = tflops_cell * cells / (conv_ms / 1e3) / 1e12
        t_peak = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        roof = {"bound": "tensor", "kernel": "conv_tc_kernel (DFT blocks on tcgen05, %s operands)"
                                             % ("BF16" if a.precision == 1 else "FP16"),
                "achieved": t_achieved, "peak": t_peak, "unit": "TFLOP/s", "frac": t_achieved / t_peak,
                "traffic": traffic, "traffic_note": traffic_note, "flops_per_cell": tflops_cell,
                "limiter": recorded_limiter(L, a.precision),
                "peak_source": "%s dense bf16 (sustained), FP16 at the same rate" % peaks_src,
                "alu_view": {"achieved": achieved, "peak": peak_alu, "frac": achieved / peak_alu,
                             "note": "FP32-equivalent transform flops (5 L log2 L + 6 L + 3 V per segment)"}}
        if rank == 0 and world == 1:
            p32 = pkg.make_params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=wl.stages,
                                  thresh=SIGMA_T[:len(wl.stages)], thresh_mode=pkg.THRESH_SIGMA,
                                  max_bins=wl.n_bins, max_candidates=1 << 20)
            with pkg.Plan(p32, device=local) as plan32:
                plan32.search(d_spec)
                c32 = [(int(c.stage), int(c.p), int(c.t)) for c in plan32.candidates()]
            plan.search(d_spec)
            ctc = [(int(c.stage), int(c.p), int(c.t)) for c in plan.candidates()]
            accuracy = tc_accuracy(wl, spec, plan, d_spec, c32, ctc)

    if rank == 0:
        cpu = None
        if world == 1 and not a.no_cpu_baseline:
            v, n, th, desc, dt = oracle_sample(wl, spec)
            cpu = {"value": v, "unit": UNIT, "cores": th, "kind": "oracle FFT route", "sample": desc,
                   "seconds": round(dt, 2)}
        phase_mean = {k: round(statistics.mean(ph[k] for ph in phases), 4) for k in phases[0]}
        srt = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": ("f32", "bf16", "f16")[a.precision],
            "data": "synthetic",
            "config": {"workload": wl.name, "n_bins": wl.n_bins, "templates": plan.info.n_templates,
                       "cells_per_step": cells, "stages": list(wl.stages), "thresh_mode": "sigma",
                       "thresh_T": list(SIGMA_T[:len(wl.stages)]), "seg_len": L, "seg_valid": V,
                       "group_size": group_size, "n_groups": plan.info.n_groups,
                       "l2": "flushed (256 MB write) before every step",
                       "parallelism": "independent spectra per rank" if world > 1 else "single GPU"},
            "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                           "min": srt[0], "max": srt[-1]},
            "phase_ms": phase_mean,
            "candidates": ncand,
            "templates_s": round(t_templates, 3),
            "roofline": roof,
            "harmonic_roofline": harm_roof,
            "plain_form_ceiling": {"value": peaks["hbm_gbs"] * 1e9 / 8.0, "unit": UNIT,
                                   "note": "unfused plane write + read, 8 B/cell at %s HBM %.1f GB/s"
                                           % (peaks_src, peaks["hbm_gbs"])},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(spec.nbytes),
                    "d2h_bytes_per_step": 8 + 24 * ncand},
            "gpu_launches": 5 * a.steps,
            "clocks": clk,
        }
        if accuracy is not None:
            line["accuracy"] = accuracy
        print(json.dumps(line))
    plan.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
