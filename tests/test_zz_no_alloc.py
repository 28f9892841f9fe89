"""The allocation-free candidate extraction, through the C ABI.

jerk_peaks_noalloc exists for callers that cannot allocate device memory at
the point where they pull candidates out (a real-time stage that reserved
its memory up front, or a program whose device memory belongs to another
allocator).  Its output must match the library's own candidate path
(jerk_search + jerk_candidates) exactly: same cells, templates and FP32
powers, in the same order, on two calls in a row (the second call reuses the
library's fixed scratch array, which still holds the first call's values).

This file is collected last so that a stop-at-first-failure run has already
run every other test; it also passes on its own in a fresh process.
"""
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


def _records(buf, n):
    from paper_1911_01353_gb300 import jerk
    raw = buf[: n * jerk.CANDIDATE_DTYPE.itemsize].cpu().numpy()
    return np.frombuffer(raw.tobytes(), dtype=jerk.CANDIDATE_DTYPE)


@pytest.mark.parametrize("thresh", [(15.0, 20.0), (6.0, 9.0)])
def test_noalloc_peaks_match_library_candidates(pkg, thresh):
    from paper_1911_01353_gb300 import jerk
    wl = synth.small_single()
    op = oracle_params(wl, thresh=thresh)
    F = wl.make()
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        plan.search(torch.from_numpy(F).cuda())
        want = plan.candidates()
        _, _, theta = plan.stats()
        cap = 1 << 16
        for call in range(2):                       # two calls in a row
            got = []
            for si, H in enumerate(op.stages):
                ptr, n_cells = plan.maxproj_ptr(si)
                out = torch.zeros(cap * jerk.CANDIDATE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
                cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
                jerk.peaks_noalloc(ptr, n_cells, float(theta[si]), H, op.zmax, op.dz, op.wmax, op.dw,
                                   out.data_ptr(), cap, cnt.data_ptr())
                torch.cuda.synchronize()
                n = int(cnt.item())
                assert 0 <= n <= cap
                got.extend(_records(out, n).tolist())
            assert len(got) == len(want) > 0
            for g, w in zip(got, want):
                p, r, t, zi, wi, stage, z, w_, power, _ = g
                assert (stage, p, t) == (w.stage, w.p, w.t)
                assert power == w.power                  # the same FP32 value
                assert (r, zi, wi, z, w_) == (w.r, w.z_idx, w.w_idx, w.z, w.w)


def test_noalloc_rejects_oversize_and_reports_full_count(pkg):
    from paper_1911_01353_gb300 import jerk
    wl = synth.small_single()
    op = oracle_params(wl, thresh=(8.0, 12.0))
    F = wl.make()
    with pkg.Plan(jerk_params(op, F.size)) as plan:
        plan.search(torch.from_numpy(F).cuda())
        ptr, n_cells = plan.maxproj_ptr(0)
        _, _, theta = plan.stats()
        out = torch.zeros(8 * jerk.CANDIDATE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        with pytest.raises(jerk.JerkError) as e:
            jerk.peaks_noalloc(ptr, (1 << 27) + 1, float(theta[0]), 1, op.zmax, op.dz, op.wmax, op.dw,
                               out.data_ptr(), 8, cnt.data_ptr())
        assert e.value.code == jerk.JERK_EINVAL
        jerk.peaks_noalloc(ptr, n_cells, float(theta[0]), 1, op.zmax, op.dz, op.wmax, op.dw,
                           out.data_ptr(), 8, cnt.data_ptr())
        torch.cuda.synchronize()
        want = [c for c in plan.candidates(cap=1 << 16) if c.stage == 1]
        assert int(cnt.item()) == len(want) > 8
        got = _records(out, 8)
        assert [int(x) for x in got["p"]] == [c.p for c in want[:8]]


def _numpy_peaks(packed: np.ndarray, theta: float):
    """The library's peak rule on a packed max-projection, in NumPy: M(p) >
    theta, M(p) > M(p-1), M(p) >= M(p+1), a missing neighbour as -inf."""
    m = (packed >> np.uint64(32)).astype(np.uint32).view(np.float32).astype(np.float64)
    left = np.concatenate([[-np.inf], m[:-1]])
    right = np.concatenate([m[1:], [-np.inf]])
    return np.nonzero((m > theta) & (m > left) & (m >= right))[0]


def _pack(vals: np.ndarray, t: np.ndarray) -> np.ndarray:
    hi = vals.astype(np.float32).view(np.uint32).astype(np.uint64) << np.uint64(32)
    return hi | (np.uint64(0xFFFFFFFF) - t.astype(np.uint64))


@pytest.mark.parametrize("n_cells,sparse", [((1 << 23) + 1234, False), (1 << 27, True)])
def test_noalloc_large_synthetic_maxproj(pkg, n_cells, sparse):
    """Sizes beyond one search of the small workload: 2^23 + 1234 cells (the
    scan gives each of its threads several blocks, and the last block is
    partial) and the largest accepted size, 2^27 cells.  A synthetic packed
    array with planted peaks, some of them carrying a template index outside
    the grid; count and records against the NumPy peak rule, two calls in a
    row."""
    from paper_1911_01353_gb300 import jerk
    zmax, dz, wmax, dw = 20, 2, 60, 20
    nz, T = 21, 147
    rng = np.random.default_rng(n_cells)
    if sparse:
        vals = np.zeros(n_cells, dtype=np.float32)
        t = np.zeros(n_cells, dtype=np.int64)
    else:
        vals = rng.uniform(0.0, 10.0, n_cells).astype(np.float32)
        t = rng.integers(0, T, n_cells)
    peaks = np.unique(np.concatenate([rng.integers(0, n_cells, 5000), [0, 1, n_cells - 2, n_cells - 1]]))
    vals[peaks] = rng.uniform(20.0, 60.0, peaks.size).astype(np.float32)
    vals[peaks[1::7]] = vals[np.minimum(peaks[1::7] + 1, n_cells - 1)]    # some plateaus
    t[peaks] = rng.integers(0, T, peaks.size)
    t[peaks[::11]] = T + 5                                                 # off the grid
    packed = _pack(vals, t)
    theta = 15.0
    want = _numpy_peaks(packed, theta)
    assert want.size > 1000
    d = torch.from_numpy(packed.view(np.int64)).cuda()
    cap = want.size + 16
    for call in range(2):
        out = torch.zeros(cap * jerk.CANDIDATE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        jerk.peaks_noalloc(d.data_ptr(), n_cells, theta, 2, zmax, dz, wmax, dw, out.data_ptr(), cap,
                           cnt.data_ptr())
        torch.cuda.synchronize()
        assert int(cnt.item()) == want.size, call
        got = _records(out, want.size)
        assert np.array_equal(got["p"], want)
        tw = t[want]
        on = tw < T
        assert np.array_equal(got["t"], tw)
        assert np.array_equal(got["power"], vals[want])
        assert np.array_equal(got["z_idx"][on], tw[on] % nz)
        assert np.array_equal(got["w_idx"][on], tw[on] // nz)
        assert np.all(got["z_idx"][~on] == -1) and np.all(got["w_idx"][~on] == -1)
        assert np.all(got["z"][~on] == 0) and np.all(got["w"][~on] == 0)
        assert np.array_equal(got["z"][on], (-zmax + (tw[on] % nz) * dz).astype(np.float32))
        assert np.all(got["stage"] == 2) and np.array_equal(got["r"], want / 2.0)
    del d
    torch.cuda.empty_cache()
