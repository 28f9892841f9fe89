"""The C ABI: the library builds for sm_103a, loads, and exports every
function ``include/jerk.h`` declares; argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1911_01353_gb300 import build, jerk
    build.build()
    return jerk.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "jerk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jerk_[a-z_]+)\s*\(", src)))


def test_header_declares_the_path():
    fns = header_functions()
    for name in ("jerk_plan_create", "jerk_templates", "jerk_search", "jerk_candidates",
                 "jerk_plan_destroy", "jerk_status_str"):
        assert name in fns


def test_library_exports_every_declared_function(L):
    from paper_1911_01353_gb300 import jerk
    fns = header_functions()
    assert sorted(jerk.EXPORTS) == fns
    for name in fns:
        assert hasattr(L, name), name


def test_checked_build_compiles_and_exports_every_declared_function():
    """The debug build (-DJERK_CHECKS, bounds checks in the kernels) compiles
    from the same sources into its own library and exports the same ABI."""
    from paper_1911_01353_gb300 import build
    path = build.build(checks=True)
    assert path == build.LIB_CHECKS and path != build.LIB
    Lc = ctypes.CDLL(path)
    for name in header_functions():
        assert hasattr(Lc, name), name


def test_status_strings(L):
    for code in range(7):
        s = L.jerk_status_str(code).decode()
        assert s.startswith("JERK_")
    assert b"unknown" in L.jerk_status_str(99)


INVALID = [("dz", 0), ("zmax", 21), ("numbetween", 4), ("pad_bins", 0), ("seg_len", 3000),
           ("seg_len", 16384), ("n_stages", 0), ("n_stages", 5), ("norm_block", 5000), ("precision", 3),
           ("precision", -1), ("max_bins", 0), ("max_bins", (1 << 29) + 1), ("max_candidates", 0),
           ("max_batch", -1), ("thresh_mode", 7), ("zmax", 4098), ("wmax", 32780), ("group_size", -1),
           ("group_size", 65537)]


def test_valid_params_accepted_without_gpu(L):
    """The validation itself (no device involved) accepts the parameter sets
    the tests and the benchmark use, including the reduced-precision filters."""
    from paper_1911_01353_gb300 import jerk
    for kw in (dict(), dict(precision=1), dict(precision=2, seg_len=4096), dict(seg_len=8192), dict(group_size=1),
               dict(group_size=65536),
               dict(stages=(1, 2, 4, 8), thresh=(1, 1, 1, 1)), dict(stages=(1, 3), thresh=(1, 1))):
        p = jerk.make_params(20, 2, 60, 20, **kw)
        assert L.jerk_params_validate(ctypes.byref(p)) == jerk.JERK_OK, kw
    p = jerk.make_params(200, 2, 600, 20, stages=(1, 2, 4, 8), thresh=(19, 17, 15, 14),
                         thresh_mode=jerk.THRESH_SIGMA, max_bins=1 << 22)
    assert L.jerk_params_validate(ctypes.byref(p)) == jerk.JERK_OK


@pytest.mark.parametrize("field,value", INVALID)
def test_invalid_params_rejected_without_gpu(L, field, value):
    """Each invalid field is rejected by the validation alone (no device), and
    jerk_plan_create then fails and leaves the handle NULL."""
    from paper_1911_01353_gb300 import jerk
    p = jerk.make_params(20, 2, 60, 20)
    assert L.jerk_params_validate(ctypes.byref(p)) == jerk.JERK_OK
    setattr(p, field, value)
    assert L.jerk_params_validate(ctypes.byref(p)) == jerk.JERK_EINVAL
    h = ctypes.c_void_p(123)
    assert L.jerk_plan_create(ctypes.byref(p), 0, ctypes.byref(h)) == jerk.JERK_EINVAL
    assert h.value is None


def test_tensor_core_filter_needs_its_segment_length(L):
    from paper_1911_01353_gb300 import jerk
    p = jerk.make_params(20, 2, 60, 20, precision=2, seg_len=2048)
    assert L.jerk_params_validate(ctypes.byref(p)) == jerk.JERK_EINVAL


def test_bad_stage_lists_rejected(L):
    from paper_1911_01353_gb300 import jerk
    for stages in ((2,), (1, 1), (1, 4, 2), (1, 16)):
        p = jerk.make_params(20, 2, 60, 20, stages=stages, thresh=(1, 1, 1, 1))
        h = ctypes.c_void_p()
        assert L.jerk_params_validate(ctypes.byref(p)) == jerk.JERK_EINVAL
        assert L.jerk_plan_create(ctypes.byref(p), 0, ctypes.byref(h)) == jerk.JERK_EINVAL


def test_null_handles(L):
    from paper_1911_01353_gb300 import jerk
    assert L.jerk_plan_destroy(None) == jerk.JERK_OK
    assert L.jerk_search(None, None, 0, None) == jerk.JERK_EINVAL
    n = ctypes.c_int64()
    assert L.jerk_candidates(None, None, 0, ctypes.byref(n)) == jerk.JERK_EINVAL
    assert L.jerk_plan_create(None, 0, None) == jerk.JERK_EINVAL
    assert L.jerk_params_validate(None) == jerk.JERK_EINVAL
