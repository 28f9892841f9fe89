"""The debug build's bounds checks (jerk_check_counts): searches, batches,
sub-grid batches, searches split by template range and plane rows of both
filters, run through the library
built with -DJERK_CHECKS, make no out-of-range global store or copy, and give
the same candidates and plane rows as the release library.  The release
library reports its checks absent."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HELPER = os.path.join(ROOT, "tests", "checks_run.py")


def run(checks):
    env = dict(os.environ)
    env["JERK_CHECKS"] = "1" if checks else "0"
    r = subprocess.run([sys.executable, HELPER], capture_output=True, text=True, timeout=900, cwd=ROOT,
                       env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_is_clean_and_equal():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chk = run(True)
    rel = run(False)
    for c in chk["checks"]:
        assert c["enabled"], c
        assert c["violations"] == 0, c
    for c in rel["checks"]:
        assert not c["enabled"] and c["violations"] == 0, c
    assert chk["runs"].keys() == rel["runs"].keys()
    for name in chk["runs"]:
        assert chk["runs"][name] == rel["runs"][name], name
    assert chk["runs"]["search0"], "the workload has candidates"
    for prec in (0, 2):
        assert chk["runs"]["split%d" % prec] == chk["runs"]["search%d" % prec], prec
