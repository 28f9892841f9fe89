"""Continuous-batching search server over one resident template bank.

A request is a spectrum plus its search range (zmax, wmax); requests arrive
over time.  The server builds ONE template bank, for the largest range it
serves, and keeps it on the device.  Each request is searched over its own
sub-grid |z| <= zmax, |w| <= wmax of that bank (jerk_search_batch_grid): the
filters of Sec. 2 depend only on (z, w), so a sub-grid of the large bank is
the smaller search.

Workers are plans sharing the bank (jerk_plan_share), each with its own
workspace, so several batches are on the GPU at once.  The loop:

* admission -- an arrived request is admitted once its spectrum fits in free
  device memory above a reserve; its spectrum is then copied to the device on
  a copy stream and stays there until its result is read;
* dispatch -- an idle worker takes admitted requests and launches them as
  one batch, whatever their lengths and ranges.  Small requests (few
  template-bins) go first, batched together, on the worker's high-priority
  stream: their blocks are scheduled ahead of the remaining blocks of large
  batches already running, so work that arrives while others run joins the
  GPU at block granularity instead of queueing behind them.  Large requests
  go first come, first served, at most `max_large` batches at a time, so
  workers stay free for small work;
* completion -- finished batches are found with CUDA events (no blocking), the
  candidates are split per request and its device memory is released.

Each request's candidates are exactly those it gets searched alone on the same
bank (tests/test_gpu_serve.py checks this for mixed ranges, lengths and arrival
times).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import jerk


@dataclass
class Request:
    rid: int
    spectrum: object                  # complex64 host array (numpy or pinned torch tensor)
    zmax: int
    wmax: int
    arrival: float = 0.0              # seconds from the start of the run
    admitted: float = -1.0
    dispatched: float = -1.0
    done: float = -1.0
    candidates: list = field(default_factory=list)   # (stage, p, t, power)
    stats: tuple = ()
    dev: object = None                # device copy while admitted
    copied: object = None             # event: device copy complete

    @property
    def n(self) -> int:
        return int(self.spectrum.shape[0])

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def templates_in(zmax: int, wmax: int, dz: int, dw: int) -> int:
    return (2 * zmax // dz + 1) * (2 * wmax // dw + 1)


def cells_of(r: Request, dz: int, dw: int, b: int = 2) -> int:
    """Template-bins of one request: b n cells times its templates."""
    return b * r.n * templates_in(r.zmax, r.wmax, dz, dw)


# -- policies (host logic, no device calls) ----------------------------------

def admissible(n_bins: int, free_bytes: int, reserve: int) -> bool:
    """A spectrum of n_bins complex64 bins may be made resident."""
    return free_bytes - 8 * n_bins >= reserve


def pick_batch(waiting, max_bins: int, max_batch: int, max_cells=None, cost=None):
    """First come, first served: the longest prefix of `waiting` that fits
    max_bins bins, max_batch spectra and (if given) max_cells of cost(r); the
    first request is taken whenever it fits max_bins on its own."""
    batch, tot, cells = [], 0, 0
    for r in waiting:
        c = cost(r) if max_cells is not None else 0
        if len(batch) == max_batch or tot + r.n > max_bins or (batch and max_cells is not None
                                                               and cells + c > max_cells):
            break
        batch.append(r)
        tot += r.n
        cells += c
    return batch


def next_batch(admitted, cost, small_cells, max_bins, max_batch, large_busy, max_large, fifo=False):
    """The batch an idle worker takes, and whether it is small.

    fifo: the oldest requests, whatever their size (the plain form uses this
    with max_batch 1).  Otherwise small requests (cost <= small_cells) go
    first, batched up to 2 small_cells of work, so they never queue behind a
    large one; then the oldest large requests, while fewer than max_large
    large batches are running (the other workers stay free for small work)."""
    if fifo:
        return pick_batch(admitted, max_bins, max_batch), False
    small = [r for r in admitted if cost(r) <= small_cells]
    if small:
        return pick_batch(small, max_bins, max_batch, 2 * small_cells, cost), True
    if large_busy >= max_large:
        return [], False
    return pick_batch(admitted, max_bins, max_batch, 0, cost), False


class Worker:
    """A plan over the shared bank, its two streams and the batch in flight."""

    def __init__(self, plan, device):
        import torch
        self.plan = plan
        self.hi = torch.cuda.Stream(device=device, priority=-1)
        self.lo = torch.cuda.Stream(device=device, priority=0)
        self.batch = []
        self.event = None
        self.small = False            # the batch in flight is small work (high-priority stream)

    @property
    def idle(self) -> bool:
        return not self.batch


class Server:
    """Serves requests with zmax <= bank zmax, wmax <= bank wmax."""

    def __init__(self, zmax, wmax, dz=2, dw=20, stages=(1,), thresh=(8.0,), thresh_mode=jerk.THRESH_SIGMA,
                 n_workers=4, worker_bins=1 << 24, max_batch=32, max_candidates=1 << 20, device=0,
                 reserve_bytes=4 << 30, small_cells=2e10, max_large=2, seg_len=0, precision=0):
        import torch
        self.torch = torch
        self.device = device
        self.dz, self.dw = dz, dw
        self.reserve = reserve_bytes
        self.small_cells = small_cells
        torch.cuda.set_device(device)
        p = jerk.make_params(zmax, dz, wmax, dw, stages=stages, thresh=thresh, thresh_mode=thresh_mode,
                             seg_len=seg_len, max_bins=worker_bins, max_candidates=max_candidates,
                             max_batch=max_batch, precision=precision)
        self.params = p
        self.bank = jerk.Plan(p, device=device)                      # builds the bank
        torch.cuda.synchronize(device)
        plans = [self.bank] + [self.bank.share(p) for _ in range(n_workers - 1)]
        self.workers = [Worker(pl, device) for pl in plans]
        self.copy_stream = torch.cuda.Stream(device=device)
        self.max_bins, self.max_batch = worker_bins, max_batch
        self.n_active, self.batch_limit = len(self.workers), max_batch
        self.max_large, self.fifo = max_large, False
        self.pending = []             # arrived or future, not admitted
        self.admitted = []            # resident, waiting for a worker
        self.finished = []
        self.t0 = None

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def _cells(self, r):
        return cells_of(r, self.dz, self.dw)

    # -- the loop ---------------------------------------------------------
    def _admit(self):
        torch = self.torch
        now = self.now()
        while self.pending and self.pending[0].arrival <= now:
            r = self.pending[0]
            free, _ = torch.cuda.mem_get_info(self.device)
            if not admissible(r.n, free, self.reserve):
                break                                  # first come, first served: wait for memory
            self.pending.pop(0)
            src = r.spectrum if isinstance(r.spectrum, torch.Tensor) else torch.from_numpy(r.spectrum)
            with torch.cuda.stream(self.copy_stream):
                r.dev = torch.empty(r.n, dtype=torch.complex64, device=self.device)
                r.dev.copy_(src, non_blocking=True)
            r.copied = torch.cuda.Event()
            r.copied.record(self.copy_stream)
            r.admitted = self.now()
            self.admitted.append(r)

    def _dispatch(self):
        active = self.workers[:self.n_active]
        for w in active:
            if not self.admitted:
                return
            if not w.idle:
                continue
            large_busy = sum(1 for x in active if not x.idle and not x.small)
            batch, small = next_batch(self.admitted, self._cells, self.small_cells, self.max_bins,
                                      self.batch_limit, large_busy, self.max_large, self.fifo)
            if not batch:
                if self.admitted[0].n > self.max_bins:
                    raise ValueError("request of %d bins exceeds the worker capacity" % self.admitted[0].n)
                return
            taken = set(id(r) for r in batch)
            self.admitted = [r for r in self.admitted if id(r) not in taken]
            st = w.hi if small else w.lo
            w.small = small
            for r in batch:
                st.wait_event(r.copied)
                r.dev.record_stream(st)
                r.dispatched = self.now()
            w.plan.search_batch([r.dev for r in batch], stream=st, zmax=[r.zmax for r in batch],
                                wmax=[r.wmax for r in batch], transient=True)
            w.event = self.torch.cuda.Event()
            w.event.record(st)
            w.batch = batch

    def _complete(self):
        for w in self.workers:
            if w.idle or not w.event.query():
                continue
            recs = w.plan.candidates()
            t = self.now()
            for i, r in enumerate(w.batch):
                r.candidates = [(c.stage, c.p, c.t, c.power) for c in recs if c.item == i]
                r.stats = w.plan.stats(i)
                r.done = t
                r.dev = None
                self.finished.append(r)
            w.batch = []

    def run(self, requests, n_workers=None, max_batch=None, fifo=False, idle_sleep=2e-4):
        """Serve `requests` (arrival times in seconds from now); returns them
        in completion order.  n_workers / max_batch / fifo restrict this run
        (one worker, batches of one, first come first served: the plain form,
        one request at a time)."""
        self.fifo = fifo
        self.n_active = len(self.workers) if n_workers is None else max(1, min(n_workers, len(self.workers)))
        self.batch_limit = self.max_batch if max_batch is None else max(1, min(max_batch, self.max_batch))
        self.t0 = time.perf_counter()
        self.finished = []
        self.pending = sorted(requests, key=lambda r: r.arrival)
        total = len(requests)
        while len(self.finished) < total:
            self._admit()
            self._dispatch()
            self._complete()
            if idle_sleep:
                time.sleep(idle_sleep)
        return self.finished

    def alone(self, r: Request):
        """The request searched by itself on the bank (reference for the mix)."""
        torch = self.torch
        src = r.spectrum if isinstance(r.spectrum, torch.Tensor) else torch.from_numpy(r.spectrum)
        x = src.to(self.device)
        pl = self.workers[0].plan
        pl.search_batch([x], zmax=[r.zmax], wmax=[r.wmax])
        recs = pl.candidates()
        return [(c.stage, c.p, c.t, c.power) for c in recs], pl.stats(0)

    def close(self):
        for w in self.workers:
            w.plan.close()


def poisson_trace(rate, duration, seed, n_range=(1 << 18, 1 << 23), zmaxes=(50, 100, 200, 300),
                  wmaxes=(0, 300, 600, 900)):
    """Arrival times (Poisson, `rate` per second over `duration` s), lengths
    log-uniform in n_range, ranges uniform over the given sets."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        n = int(2.0 ** rng.uniform(np.log2(n_range[0]), np.log2(n_range[1])))
        out.append((t, n, int(rng.choice(zmaxes)), int(rng.choice(wmaxes))))


def summary(done, dz, dw):
    """Throughput (template-bins/s) and latency percentiles of a finished run."""
    lat = np.array([r.latency for r in done])
    span = max(r.done for r in done) - min(r.arrival for r in done)
    cells = sum(cells_of(r, dz, dw) for r in done)
    return {"requests": len(done), "cells": int(cells), "seconds": span, "cells_per_s": cells / span,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
