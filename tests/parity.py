"""Helpers for the GPU-vs-oracle parity tests (test code, no method arithmetic
beyond reading the oracle's outputs)."""
from __future__ import annotations

import numpy as np

# |P_gpu - P_oracle| <= PLANE_TOL * max P_oracle for every plane cell and every
# max-projection value.
PLANE_TOL = 1e-4


def lib_ready():
    """Build libjerk.so (no-op when current) and return the package."""
    from paper_1911_01353_gb300 import build
    build.build()
    import paper_1911_01353_gb300 as pkg
    return pkg


def oracle_params(wl, mode="abs", thresh=None, pad=16, norm_block=1024):
    import oracle
    return oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=tuple(wl.stages),
                         thresh_mode=mode, thresh=tuple(thresh or wl.thresh), pad_bins=pad,
                         norm_block=norm_block)


def jerk_params(op, n_bins, seg_len=0, max_candidates=1 << 16):
    from paper_1911_01353_gb300 import jerk
    return jerk.make_params(op.zmax, op.dz, op.wmax, op.dw, stages=op.stages, thresh=op.thresh,
                            thresh_mode=jerk.THRESH_SIGMA if op.thresh_mode == "sigma" else jerk.THRESH_ABS,
                            pad_bins=op.pad_bins, seg_len=seg_len, norm_block=op.norm_block,
                            max_bins=n_bins, max_candidates=max_candidates)


def runner_up_margin(S: np.ndarray) -> np.ndarray:
    """Per cell, best minus second-best S over templates (FP64)."""
    if S.shape[0] < 2:
        return np.full(S.shape[1], np.inf)
    part = np.partition(S, S.shape[0] - 2, axis=0)
    return part[-1] - part[-2]


def compare_maxproj(M_gpu, t_gpu, M_or, t_or, S_or, tol_abs):
    """Values within tol_abs everywhere; argmax equal wherever the oracle's
    best and runner-up differ by more than 2 tol_abs.  Returns the number of
    cells excluded from the argmax comparison."""
    assert M_gpu.shape == M_or.shape
    err = np.abs(M_gpu.astype(np.float64) - M_or.astype(np.float64))
    assert float(err.max()) <= tol_abs, "max-projection error %g > %g" % (err.max(), tol_abs)
    margin = runner_up_margin(S_or)
    sure = margin > 2 * tol_abs
    bad = np.nonzero(sure & (t_gpu != t_or))[0]
    assert bad.size == 0, "argmax differs at %s" % bad[:10]
    return int((~sure).sum())


def compare_candidates(gpu, res, tol_abs):
    """GPU candidates (records) vs the oracle's result.  A cell is guarded
    (left out of the exact comparison) when one of its decisions -- above
    threshold, above the left neighbour, not below the right one, the
    argmax -- is within 2 tol_abs of flipping in the oracle.  Returns the
    number of guarded cells among the candidates of either side."""
    got = {(int(c.stage), int(c.p)): (int(c.t), float(c.power)) for c in gpu}
    want = {(c[0], c[1]): (c[2], c[3]) for c in res.candidates}
    guarded = 0
    for H in res.maxproj:
        M, arg = res.maxproj[H]
        fund, S = res.sums[H]
        th = float(res.theta[H])
        keys = {p for (h, p) in list(got) + list(want) if h == H}
        for p in keys:
            m = float(M[p])
            l = float(M[p - 1]) if p > 0 else -np.inf
            r = float(M[p + 1]) if p + 1 < M.size else -np.inf
            col = np.sort(S[:, p])
            second = col[-2] if col.size > 1 else -np.inf
            near = (abs(m - th) <= 2 * tol_abs or abs(m - l) <= 2 * tol_abs or
                    abs(m - r) <= 2 * tol_abs or col[-1] - second <= 2 * tol_abs)
            if near:
                guarded += 1
                continue
            assert (H, p) in got, "oracle candidate (H=%d, p=%d) missing on GPU" % (H, p)
            assert (H, p) in want, "GPU candidate (H=%d, p=%d) not an oracle candidate" % (H, p)
            assert got[(H, p)][0] == want[(H, p)][0], "template differs at (H=%d, p=%d)" % (H, p)
            assert abs(got[(H, p)][1] - want[(H, p)][1]) <= tol_abs
    return guarded
