"""The filter kernels' register DFTs (csrc/fft.cuh: dft16, dft8, dft4 with the
eighth-root twiddles formed inside their butterflies) compiled as host code
and checked against a direct DFT in FP64 -- no GPU needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include <cstdio>
#include "fft.cuh"
using namespace jerk;
template <int SIGN, int N, class F> void run(F f) {
    unsigned s = 12345u + 77u * N + (SIGN > 0);
    for (int rep = 0; rep < 64; ++rep) {
        float2 a[N];
        for (int k = 0; k < N; ++k) {
            s = s * 1664525u + 1013904223u; float re = (float)(s >> 8) / 16777216.0f - 0.5f;
            s = s * 1664525u + 1013904223u; float im = (float)(s >> 8) / 16777216.0f - 0.5f;
            a[k] = make_float2(re, im);
            printf("%d %d %d %d %.9e %.9e\n", SIGN, N, rep, k, re, im);
        }
        f(a);
        for (int k = 0; k < N; ++k) printf("%d %d %d %d %.9e %.9e\n", SIGN, N, rep, N + k, a[k].x, a[k].y);
    }
}
int main() {
    run<+1, 16>([](float2 (&a)[16]) { dft16<+1>(a); });
    run<-1, 16>([](float2 (&a)[16]) { dft16<-1>(a); });
    run<+1, 8>([](float2 (&a)[8]) { dft8<+1>(a); });
    run<-1, 8>([](float2 (&a)[8]) { dft8<-1>(a); });
    run<+1, 4>([](float2 (&a)[4]) { dft4<+1>(a[0], a[1], a[2], a[3]); });
    run<-1, 4>([](float2 (&a)[4]) { dft4<-1>(a[0], a[1], a[2], a[3]); });
    return 0;
}
'''


def test_register_dfts_match_direct_dft(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "dft_blocks.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "dft_blocks"
    subprocess.check_call([nvcc, "-std=c++17", "-x", "cu", "-I", os.path.join(ROOT, "paper_1911_01353_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                          stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    rows = np.array([list(map(float, line.split())) for line in out.splitlines()])
    checked = 0
    for sign in (1, -1):
        for n in (16, 8, 4):
            sel = rows[(rows[:, 0] == sign) & (rows[:, 1] == n)]
            for rep in np.unique(sel[:, 2]):
                blk = sel[sel[:, 2] == rep]
                blk = blk[np.argsort(blk[:, 3])]
                x = blk[:n, 4] + 1j * blk[:n, 5]
                y = blk[n:, 4] + 1j * blk[n:, 5]
                k = np.arange(n)
                want = np.exp(sign * 2j * np.pi * np.outer(k, k) / n) @ x
                assert np.max(np.abs(y - want)) <= 2e-6 * max(1.0, np.max(np.abs(want))), (sign, n, rep)
                checked += 1
    assert checked == 2 * 3 * 64
