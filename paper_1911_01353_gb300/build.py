"""Build libjerk.so (sm_103a) in-tree with nvcc.

Every translation unit is compiled in parallel, then linked into
``paper_1911_01353_gb300/_build/libjerk.so``.  Usage:
``python -m paper_1911_01353_gb300.build [--force] [--checks]``.

``--checks`` builds the debug library instead,
``paper_1911_01353_gb300/_build_checks/libjerk.so``, compiled with
-DJERK_CHECKS: its kernels check the indices of their global stores and
copies and count violations (``jerk_check_counts``).  The Python binding
loads it when JERK_CHECKS=1.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libjerk.so")
OUT_CHECKS = os.path.join(HERE, "_build_checks")
LIB_CHECKS = os.path.join(OUT_CHECKS, "libjerk.so")
SOURCES = ["plan.cu", "templates.cu", "conv.cu", "conv_tc.cu", "kernels.cu", "noalloc.cu", "refine.cu",
           "subharmonic.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libjerk.so")


def _deps(src: str):
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "jerk.h")]


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    out, lib = (OUT_CHECKS, LIB_CHECKS) if checks else (OUT, LIB)
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    newest = max(os.path.getmtime(p) for p in _deps(""))
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    objs = []
    extra = ["-DJERK_CHECKS"] if checks else []

    def compile_one(src):
        obj = os.path.join(out, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for obj, log in ex.map(compile_one, SOURCES):
            objs.append(obj)
            if verbose and log:
                sys.stderr.write(log)
    tmp = lib + ".tmp%d" % os.getpid()
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checks="--checks" in sys.argv))
