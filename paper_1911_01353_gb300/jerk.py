"""ctypes binding of libjerk.so (argument marshalling only).

Every step of the search runs in the library's CUDA kernels; this module only
converts Python/PyTorch arguments into the C ABI declared in
``include/jerk.h``.  PyTorch supplies device memory and streams.  If the
library is missing the import of ``lib()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libjerk.so")
# the debug build with bounds checks in its kernels (see jerk_check_counts)
LIB_CHECKS_PATH = os.path.join(_HERE, "_build_checks", "libjerk.so")

JERK_OK, JERK_EINVAL, JERK_ENOMEM, JERK_ECUDA, JERK_ETIMEOUT, JERK_EOVERFLOW, JERK_ESTATE = range(7)
THRESH_ABS, THRESH_SIGMA = 0, 1

# Every function the header declares (kept in step with include/jerk.h).
EXPORTS = ("jerk_plan_create", "jerk_templates", "jerk_search", "jerk_search_host", "jerk_search_batch",
           "jerk_candidates", "jerk_plan_destroy", "jerk_status_str", "jerk_plan_info",
           "jerk_normalise", "jerk_taps", "jerk_plane", "jerk_maxproj", "jerk_stats",
           "jerk_profile", "jerk_phase_times", "jerk_peaks_noalloc", "jerk_template_row",
           "jerk_search_batch_grid", "jerk_plan_share", "jerk_power_at", "jerk_refine", "jerk_check_waits",
           "jerk_measure_peaks", "jerk_measure_packed_fma", "jerk_check_counts", "jerk_check_inject",
           "jerk_params_validate", "jerk_search_range", "jerk_range_sums", "jerk_select", "jerk_subharmonic")
PHASES = ("normalise", "conv", "harmonic", "stats", "peaks")


class Params(ctypes.Structure):
    _fields_ = [("zmax", ctypes.c_int32), ("dz", ctypes.c_int32),
                ("wmax", ctypes.c_int32), ("dw", ctypes.c_int32),
                ("numbetween", ctypes.c_int32), ("pad_bins", ctypes.c_int32),
                ("seg_len", ctypes.c_int32), ("n_stages", ctypes.c_int32),
                ("stages", ctypes.c_int32 * 4), ("thresh_mode", ctypes.c_int32),
                ("thresh", ctypes.c_float * 4), ("norm_block", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_bins", ctypes.c_int64),
                ("max_candidates", ctypes.c_int64), ("max_batch", ctypes.c_int32),
                ("group_size", ctypes.c_int32)]


class Candidate(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int64), ("r", ctypes.c_double), ("t", ctypes.c_int32),
                ("z_idx", ctypes.c_int32), ("w_idx", ctypes.c_int32), ("stage", ctypes.c_int32),
                ("z", ctypes.c_float), ("w", ctypes.c_float), ("power", ctypes.c_float),
                ("item", ctypes.c_int32)]


class Refined(ctypes.Structure):
    _fields_ = [("r", ctypes.c_double), ("z", ctypes.c_float), ("w", ctypes.c_float),
                ("power", ctypes.c_float), ("power_in", ctypes.c_float), ("is_peak", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int32), ("nw", ctypes.c_int32), ("n_templates", ctypes.c_int32),
                ("bank_halfwidth", ctypes.c_int32), ("taps", ctypes.c_int32),
                ("seg_len", ctypes.c_int32), ("seg_valid", ctypes.c_int32), ("device", ctypes.c_int32),
                ("max_bins", ctypes.c_int64), ("slot_floats", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("transforms", ctypes.c_int64),
                ("n_groups", ctypes.c_int32), ("reserved", ctypes.c_int32), ("d_bank", ctypes.c_void_p),
                ("bank_bytes", ctypes.c_int64)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libjerk.so (built by ``paper_1911_01353_gb300.build``)."""
    global _lib
    if _lib is None:
        checks = os.environ.get("JERK_CHECKS") == "1"
        path = LIB_CHECKS_PATH if checks else LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError("libjerk.so is not built (%s); run "
                               "`python -m paper_1911_01353_gb300.build%s`" % (path, " --checks" if checks else ""))
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        st = ctypes.c_int
        sig = {
            "jerk_plan_create": ([ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(vp)], st),
            "jerk_params_validate": ([ctypes.POINTER(Params)], st),
            "jerk_search_range": ([vp, vp, i64, i32, i32, vp], st),
            "jerk_subharmonic": ([vp, vp, i64, i32, vp, vp, vp], st),
            "jerk_range_sums": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)], st),
            "jerk_select": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), vp], st),
            "jerk_templates": ([vp, vp], st),
            "jerk_search": ([vp, vp, i64, vp], st),
            "jerk_search_host": ([vp, vp, i64, vp], st),
            "jerk_search_batch": ([vp, ctypes.POINTER(vp), ctypes.POINTER(i64), i32, i32, vp], st),
            "jerk_candidates": ([vp, ctypes.POINTER(Candidate), i64, ctypes.POINTER(i64)], st),
            "jerk_plan_destroy": ([vp], st),
            "jerk_status_str": ([st], ctypes.c_char_p),
            "jerk_plan_info": ([vp, ctypes.POINTER(Info)], st),
            "jerk_normalise": ([vp, vp, i64, vp, vp], st),
            "jerk_taps": ([vp, i32, i32, vp, vp], st),
            "jerk_plane": ([vp, vp, i64, i32, i32, vp, vp], st),
            "jerk_maxproj": ([vp, i32, i32, ctypes.POINTER(vp), ctypes.POINTER(i64)], st),
            "jerk_stats": ([vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_float)], st),
            "jerk_profile": ([vp, i32], st),
            "jerk_phase_times": ([vp, ctypes.POINTER(ctypes.c_float), i32], st),
            "jerk_peaks_noalloc": ([vp, i64, ctypes.c_float, i32, i32, i32, i32, i32, vp, i64, vp, vp], st),
            "jerk_template_row": ([vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)], st),
            "jerk_search_batch_grid": ([vp, ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                        ctypes.POINTER(i32), i32, i32, vp], st),
            "jerk_plan_share": ([vp, ctypes.POINTER(Params), ctypes.POINTER(vp)], st),
            "jerk_power_at": ([vp, vp, i64, ctypes.POINTER(ctypes.c_double), i64, ctypes.POINTER(ctypes.c_float), vp],
                              st),
            "jerk_refine": ([vp, vp, i64, ctypes.POINTER(Candidate), i32, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(i32), ctypes.POINTER(Refined), vp], st),
            "jerk_check_counts": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32)], st),
            "jerk_check_inject": ([vp, i32, i32], st),
            "jerk_check_waits": ([vp, i32, vp], st),
            "jerk_measure_peaks": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                                   st),
            "jerk_measure_packed_fma": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double)], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def measure_peaks(device: int = 0):
    """(FP32 TFLOP/s, L2 read GB/s) measured on `device` (jerk_measure_peaks)."""
    f, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().jerk_measure_peaks(device, ctypes.byref(f), ctypes.byref(b)), "jerk_measure_peaks")
    return f.value, b.value


def measure_packed_fma(device: int = 0):
    """FP32 TFLOP/s of packed (f32x2) FMAs measured on `device` (jerk_measure_packed_fma)."""
    f = ctypes.c_double()
    _check(lib().jerk_measure_packed_fma(device, ctypes.byref(f)), "jerk_measure_packed_fma")
    return f.value


class JerkError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s: %s" % (what, lib().jerk_status_str(code).decode()))


def _check(code: int, what: str):
    if code != JERK_OK:
        raise JerkError(code, what)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_params(zmax, dz, wmax, dw, stages=(1, 2), thresh=(15.0, 20.0), thresh_mode=THRESH_ABS,
                pad_bins=16, seg_len=0, norm_block=1024, max_bins=1 << 16, max_candidates=1 << 16,
                numbetween=2, precision=0, max_batch=1, group_size=0) -> Params:
    p = Params()
    p.zmax, p.dz, p.wmax, p.dw = zmax, dz, wmax, dw
    p.numbetween, p.pad_bins, p.seg_len = numbetween, pad_bins, seg_len
    p.n_stages = len(stages)
    for i in range(4):
        p.stages[i] = stages[i] if i < len(stages) else 0
        p.thresh[i] = thresh[i] if i < len(thresh) else 0.0
    p.thresh_mode = thresh_mode
    p.norm_block, p.precision = norm_block, precision
    p.max_bins, p.max_candidates = max_bins, max_candidates
    p.max_batch, p.group_size = max_batch, group_size
    return p


CANDIDATE_DTYPE = np.dtype([("p", "<i8"), ("r", "<f8"), ("t", "<i4"), ("z_idx", "<i4"), ("w_idx", "<i4"),
                            ("stage", "<i4"), ("z", "<f4"), ("w", "<f4"), ("power", "<f4"),
                            ("item", "<i4")])
BATCH_GRAPH = 1
BATCH_TRANSIENT = 2


def peaks_noalloc(d_maxproj: int, n_cells: int, theta: float, stage: int, zmax: int, dz: int, wmax: int,
                  dw: int, d_out: int, cap: int, d_count: int, stream=None):
    """Candidate extraction that allocates no device memory (device pointers in
    and out; see ``jerk_peaks_noalloc`` in include/jerk.h)."""
    _check(lib().jerk_peaks_noalloc(ctypes.c_void_p(d_maxproj), n_cells, theta, stage, zmax, dz, wmax, dw,
                                    ctypes.c_void_p(d_out), cap, ctypes.c_void_p(d_count),
                                    _stream_handle(stream)), "jerk_peaks_noalloc")


class Plan:
    """One search configuration on one device; owns the template bank."""

    def __init__(self, params: Params, device: int = 0, build_templates: bool = True, stream=None,
                 share_with: "Plan | None" = None):
        self.params = params
        h = ctypes.c_void_p()
        if share_with is not None:
            # the bank of `share_with`, a workspace of this plan's own
            _check(lib().jerk_plan_share(share_with._h, ctypes.byref(params), ctypes.byref(h)), "jerk_plan_share")
            device = share_with.device
            build_templates = False
        else:
            _check(lib().jerk_plan_create(ctypes.byref(params), device, ctypes.byref(h)), "jerk_plan_create")
        self._h = h
        self.device = device
        self.info = Info()
        _check(lib().jerk_plan_info(self._h, ctypes.byref(self.info)), "jerk_plan_info")
        if build_templates:
            self.templates(stream)

    # -- lifecycle --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().jerk_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the path ---------------------------------------------------------
    def templates(self, stream=None):
        _check(lib().jerk_templates(self._h, _stream_handle(stream)), "jerk_templates")

    def search(self, spec, stream=None):
        """Enqueue a search of a complex64 CUDA tensor (no host sync)."""
        assert spec.is_cuda and spec.is_contiguous() and str(spec.dtype) == "torch.complex64"
        _check(lib().jerk_search(self._h, ctypes.c_void_p(spec.data_ptr()), spec.numel(),
                                 _stream_handle(stream)), "jerk_search")

    def search_range(self, spec, t_lo: int, t_hi: int, stream=None):
        """Enqueue a partial search over templates t_lo <= t < t_hi
        (jerk_search_range); merge with the other ranges, then select()."""
        assert spec.is_cuda and spec.is_contiguous() and str(spec.dtype) == "torch.complex64"
        _check(lib().jerk_search_range(self._h, ctypes.c_void_p(spec.data_ptr()), spec.numel(), int(t_lo),
                                       int(t_hi), _stream_handle(stream)), "jerk_search_range")

    def range_sums(self):
        """(sum, sum of squares, count) per stage of the last partial search
        (jerk_range_sums); synchronises."""
        ns = int(self.params.n_stages)
        a, b, c = (ctypes.c_double * ns)(), (ctypes.c_double * ns)(), (ctypes.c_double * ns)()
        _check(lib().jerk_range_sums(self._h, a, b, c), "jerk_range_sums")
        return np.array(a[:]), np.array(b[:]), np.array(c[:])

    def select(self, sums=None, sumsq=None, counts=None, stream=None):
        """Thresholds from (reduced) sums and the peaks of the current
        max-projections (jerk_select); synchronises."""
        ns = int(self.params.n_stages)

        def arr(x):
            return None if x is None else (ctypes.c_double * ns)(*[float(v) for v in x])
        _check(lib().jerk_select(self._h, arr(sums), arr(sumsq), arr(counts), _stream_handle(stream)),
               "jerk_select")

    def search_subharmonic(self, spec, cap: int = 1 << 16, stream=None):
        """The search with the harmonic sum indexed by the highest harmonic
        (jerk_subharmonic) for every stage of the plan: the whole power plane
        (jerk_plane, n_templates x b n floats, allocated here), per stage the
        max-projection and sums of S'_H, the threshold (the plan's mode and
        values) and the peaks (jerk_peaks_noalloc).  Synchronises.  Returns
        (candidate records, [(mu, sd, theta)] per stage, [packed int64
        max-projection tensors])."""
        import torch
        n = spec.numel()
        T, bN = int(self.info.n_templates), 2 * n
        dev = torch.device("cuda", self.device)
        plane = torch.empty((T, bN), dtype=torch.float32, device=dev)
        self.plane(spec, 0, T, plane, stream=stream)
        p = self.params
        recs, stats, maxprojs = [], [], []
        for si in range(int(p.n_stages)):
            H = int(p.stages[si])
            M = torch.empty(bN, dtype=torch.int64, device=dev)
            sums = torch.zeros(2, dtype=torch.float64, device=dev)
            _check(lib().jerk_subharmonic(self._h, ctypes.c_void_p(plane.data_ptr()), n, H,
                                          ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(sums.data_ptr()),
                                          _stream_handle(stream)), "jerk_subharmonic")
            torch.cuda.synchronize(self.device)
            s1, s2 = (float(x) for x in sums.cpu())
            cnt = float(T) * float(bN)
            mu = s1 / cnt
            sd = math.sqrt(max(0.0, s2 / cnt - mu * mu))
            theta = float(np.float32(mu + float(p.thresh[si]) * sd)) if p.thresh_mode == THRESH_SIGMA \
                else float(np.float32(p.thresh[si]))
            out = torch.zeros(cap * CANDIDATE_DTYPE.itemsize, dtype=torch.uint8, device=dev)
            cnt_d = torch.zeros(1, dtype=torch.int64, device=dev)
            peaks_noalloc(M.data_ptr(), bN, theta, H, int(p.zmax), int(p.dz), int(p.wmax), int(p.dw),
                          out.data_ptr(), cap, cnt_d.data_ptr(), stream)
            torch.cuda.synchronize(self.device)
            k = int(cnt_d.item())
            if k > cap:
                raise JerkError(JERK_EOVERFLOW, "jerk_peaks_noalloc (%d found)" % k)
            raw = out[: k * CANDIDATE_DTYPE.itemsize].cpu().numpy()
            recs.extend(np.frombuffer(raw.tobytes(), dtype=CANDIDATE_DTYPE).tolist())
            stats.append((mu, sd, theta))
            maxprojs.append(M)
        return recs, stats, maxprojs

    def share(self, params: Params) -> "Plan":
        """A new plan over this plan's template bank with its own workspace
        (jerk_plan_share)."""
        return Plan(params, share_with=self)

    def search_batch(self, specs, graph: bool = False, stream=None, zmax=None, wmax=None,
                     transient: bool = False):
        """Enqueue one batched search of several complex64 CUDA tensors;
        with zmax / wmax (one value per spectrum) each spectrum is searched
        over its own sub-grid of the bank (jerk_search_batch_grid)."""
        n = len(specs)
        ptrs = (ctypes.c_void_p * n)(*[ctypes.c_void_p(s.data_ptr()) for s in specs])
        lens = (ctypes.c_int64 * n)(*[s.numel() for s in specs])
        self._batch_ref = specs
        flags = (BATCH_GRAPH if graph else 0) | (BATCH_TRANSIENT if transient else 0)
        if zmax is None and wmax is None and not transient:
            _check(lib().jerk_search_batch(self._h, ptrs, lens, n, flags, _stream_handle(stream)),
                   "jerk_search_batch")
            return
        zp = wp = None
        if zmax is not None or wmax is not None:
            zmax = [int(self.params.zmax)] * n if zmax is None else list(zmax)
            wmax = [int(self.params.wmax)] * n if wmax is None else list(wmax)
            if len(zmax) != n or len(wmax) != n:
                raise ValueError("one zmax and one wmax per spectrum")
            zp = (ctypes.c_int32 * n)(*zmax)
            wp = (ctypes.c_int32 * n)(*wmax)
        _check(lib().jerk_search_batch_grid(self._h, ptrs, lens, zp, wp, n, flags, _stream_handle(stream)),
               "jerk_search_batch_grid")

    def search_host(self, spec: np.ndarray, stream=None):
        """Enqueue a search of a host complex64 array (copied by the library)."""
        a = np.ascontiguousarray(spec, dtype=np.complex64)
        self._host_ref = a
        _check(lib().jerk_search_host(self._h, a.ctypes.data_as(ctypes.c_void_p), a.size,
                                      _stream_handle(stream)), "jerk_search_host")

    def candidates(self, cap: int | None = None):
        """Synchronise and return the candidate records (Candidate) sorted by
        (item, stage, p).  Without `cap` the count is read first and the
        buffer sized to it."""
        if cap is None:
            n = ctypes.c_int64()
            code = lib().jerk_candidates(self._h, None, 0, ctypes.byref(n))
            if code not in (JERK_OK, JERK_EOVERFLOW):
                _check(code, "jerk_candidates")
            if n.value > int(self.params.max_candidates):
                raise JerkError(JERK_EOVERFLOW, "jerk_candidates (%d found)" % n.value)
            cap = n.value
        buf = (Candidate * max(cap, 1))()
        n = ctypes.c_int64()
        code = lib().jerk_candidates(self._h, buf, cap, ctypes.byref(n))
        if code not in (JERK_OK, JERK_EOVERFLOW):
            _check(code, "jerk_candidates")
        if code == JERK_EOVERFLOW:
            raise JerkError(code, "jerk_candidates (%d found)" % n.value)
        return [buf[i] for i in range(n.value)]

    def power_at(self, spec, points, stream=None) -> np.ndarray:
        """Matched-filter power at (r, z, w) points (array of shape (n, 3)) of
        the complex64 CUDA tensor `spec` (jerk_power_at)."""
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
        out = np.empty(pts.shape[0], dtype=np.float32)
        _check(lib().jerk_power_at(self._h, ctypes.c_void_p(spec.data_ptr()), spec.numel(),
                                   pts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pts.shape[0],
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream_handle(stream)),
               "jerk_power_at")
        return out

    def refine(self, spec, cands, step, half, stream=None):
        """Refined candidates (jerk_refine): `cands` are Candidate records of
        this spectrum, step = (dr, dz, dw), half = (hr, hz, hw)."""
        n = len(cands)
        arr = (Candidate * max(n, 1))(*cands)
        out = (Refined * max(n, 1))()
        st = (ctypes.c_double * 3)(*[float(x) for x in step])
        hf = (ctypes.c_int32 * 3)(*[int(x) for x in half])
        _check(lib().jerk_refine(self._h, ctypes.c_void_p(spec.data_ptr()), spec.numel(), arr, n, st, hf, out,
                                 _stream_handle(stream)), "jerk_refine")
        return [out[i] for i in range(n)]

    def check_waits(self, limit_us: int = 20000, stream=None) -> int:
        """Status code of jerk_check_waits (JERK_ETIMEOUT when the bounded
        device wait and its error report work); argument errors raise."""
        code = int(lib().jerk_check_waits(self._h, int(limit_us), _stream_handle(stream)))
        if code == JERK_EINVAL:
            _check(code, "jerk_check_waits")
        return code

    def check_counts(self):
        """(violations, first site, compiled in) of the debug build's bounds
        checks (jerk_check_counts); waits for the plan's work."""
        v, site, on = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().jerk_check_counts(self._h, ctypes.byref(v), ctypes.byref(site), ctypes.byref(on)),
               "jerk_check_counts")
        return int(v.value), int(site.value), bool(on.value)

    def check_inject(self, mode: int, position: int = 3):
        """Set the debug build's test hook (jerk_check_inject); returns the
        status code (JERK_ESTATE from the release build)."""
        code = lib().jerk_check_inject(self._h, int(mode), int(position))
        if code == JERK_EINVAL:
            _check(code, "jerk_check_inject")
        return code

    def stats(self, item: int = 0):
        k = int(self.params.n_stages)
        mu = (ctypes.c_double * k)()
        sd = (ctypes.c_double * k)()
        th = (ctypes.c_float * k)()
        _check(lib().jerk_stats(self._h, item, mu, sd, th), "jerk_stats")
        return list(mu), list(sd), list(th)

    def template_row(self, t: int):
        """(bank row, group tap offset bM_g, group segment length V_g) of template t."""
        r, o, v = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().jerk_template_row(self._h, t, ctypes.byref(r), ctypes.byref(o), ctypes.byref(v)),
               "jerk_template_row")
        return r.value, o.value, v.value

    def profile(self, enable: bool = True):
        _check(lib().jerk_profile(self._h, 1 if enable else 0), "jerk_profile")

    def phase_times(self):
        """{phase: ms} of the last profiled search."""
        ms = (ctypes.c_float * len(PHASES))()
        _check(lib().jerk_phase_times(self._h, ms, len(PHASES)), "jerk_phase_times")
        return dict(zip(PHASES, list(ms)))

    # -- single steps -----------------------------------------------------
    def normalise(self, spec_in, spec_out, stream=None):
        _check(lib().jerk_normalise(self._h, ctypes.c_void_p(spec_in.data_ptr()), spec_in.numel(),
                                    ctypes.c_void_p(spec_out.data_ptr()), _stream_handle(stream)),
               "jerk_normalise")

    def taps(self, t0: int, nt: int, out, stream=None):
        """out: complex128 CUDA tensor [nt, K]."""
        _check(lib().jerk_taps(self._h, t0, nt, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "jerk_taps")

    def plane(self, spec, t0: int, nt: int, out, stream=None):
        """out: float32 CUDA tensor [nt, 2 n]."""
        _check(lib().jerk_plane(self._h, ctypes.c_void_p(spec.data_ptr()), spec.numel(), t0, nt,
                                ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), "jerk_plane")

    def maxproj_ptr(self, stage_idx: int, item: int = 0):
        ptr = ctypes.c_void_p()
        n = ctypes.c_int64()
        _check(lib().jerk_maxproj(self._h, item, stage_idx, ctypes.byref(ptr), ctypes.byref(n)), "jerk_maxproj")
        return ptr.value, n.value

    def maxproj_tensor(self, stage_idx: int, item: int = 0):
        """The packed stage max-projection in place on the device, as an int64
        CUDA tensor view (writable; valid until the plan's next search).  The
        packed entries are non-negative, so signed and unsigned order agree."""
        import torch
        ptr, n = self.maxproj_ptr(stage_idx, item)
        return torch.as_tensor(_DevArray(ptr, n, "<i8"), device="cuda:%d" % self.device)

    def maxproj(self, stage_idx: int, item: int = 0):
        """Copy the packed stage max-projection to host: (float32 M, int64 t)."""
        import torch
        ptr, n = self.maxproj_ptr(stage_idx, item)
        dev = torch.as_tensor(_DevArray(ptr, n, "<i8"), device="cuda:%d" % self.device)
        torch.cuda.synchronize(self.device)
        host = dev.cpu().numpy().view(np.uint64)
        M = (host >> np.uint64(32)).astype(np.uint32).view(np.float32)
        t = (np.uint64(0xFFFFFFFF) - (host & np.uint64(0xFFFFFFFF))).astype(np.int64)
        return M, t


class _DevArray:
    """A view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3}
