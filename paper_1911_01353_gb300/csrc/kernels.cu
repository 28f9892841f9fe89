// Normalisation, harmonic sum, statistics and peak finding.
#include <cfloat>

#include "device_sync.cuh"
#include "jerk_internal.h"

namespace jerk {

// ---------------------------------------------------------------------------
// Power normalisation (the paper is silent; reading): for each block of B
// bins, med = element of rank floor((n-1)/2) of |F_k|^2 (FP64, exact for
// FP32 input), F_k <- F_k (med / ln 2)^(-1/2).  One CTA per block; bitonic
// sort of the FP64 bit patterns (non-negative, so integer order = value order).
// ---------------------------------------------------------------------------
__global__ void normalise_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, int64_t n,
                                 int B, int SZ) {
    extern __shared__ unsigned long long key[];   // [SZ]
    const int64_t s0 = (int64_t)blockIdx.x * B;
    const int nb = (int)((n - s0) < B ? (n - s0) : B);
    for (int i = threadIdx.x; i < SZ; i += blockDim.x) {
        unsigned long long k = ~0ull;
        if (i < nb) {
            const float2 f = in[s0 + i];
            const double re = f.x, im = f.y;
            k = (unsigned long long)__double_as_longlong(re * re + im * im);
        }
        key[i] = k;
    }
    __syncthreads();
    for (int k = 2; k <= SZ; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < SZ; i += blockDim.x) {
                const int ixj = i ^ jj;
                if (ixj > i) {
                    const unsigned long long a = key[i], b = key[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        key[i] = b;
                        key[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    const double med = __longlong_as_double((long long)key[(nb - 1) / 2]);
    const double scale = med > 0.0 ? 1.0 / sqrt(med / 0.69314718055994530942) : 1.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const float2 f = in[s0 + i];
        out[s0 + i] = make_float2((float)((double)f.x * scale), (float)((double)f.y * scale));
    }
}

cudaError_t launch_normalise(const float2 *in, float2 *out, int64_t n, int B, cudaStream_t st) {
    int SZ = 1;
    while (SZ < B) SZ <<= 1;
    const int64_t nblk = (n + B - 1) / B;
    const size_t sm = (size_t)SZ * sizeof(unsigned long long);
    normalise_kernel<<<(unsigned)nblk, 512, sm, st>>>(in, out, n, B, SZ);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Harmonic sum (Sec. 3 names it; S_H(p, z, w) = sum_{h=1..H} P(h p, h z, h w)
// is the reading) and the stage-H max-projection over (z, w).  Each thread
// owns 4 consecutive fundamental cells p and loops over the fundamentals in
// ascending t; the harmonic rows P(h p, h z, h w) were written by the fused
// kernel into per-(h, fundamental) slots indexed by p (128-byte aligned), so
// every read is a coalesced 16-byte load.  Sums are FP32 in fixed h order;
// the max keeps the lowest t on ties.  HBM-bound: each slot float is read once.
// ---------------------------------------------------------------------------
template <int NS>
__global__ void __launch_bounds__(256, 4) harmonic_kernel(HarmArgs a, bool stats) {
    __shared__ double red[JERK_MAX_STAGES][2][8];
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    int top = 0;   // highest stage index defined at p0
#pragma unroll
    for (int si = 1; si < NS; ++si)
        if (p0 < a.n_cells[si]) top = si;
    bool ok[NS][4];
#pragma unroll
    for (int si = 1; si < NS; ++si)
#pragma unroll
        for (int c = 0; c < 4; ++c) ok[si][c] = p0 + c < a.n_cells[si];
    float mx[NS][4];
    int am[NS][4];
    double d1[NS], d2[NS];
    float c1[NS], c2[NS];
#pragma unroll
    for (int si = 0; si < NS; ++si) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            mx[si][c] = -1.0f;
            am[si][c] = 0;
        }
        d1[si] = d2[si] = 0.0;
        c1[si] = c2[si] = 0.f;
    }
    int hlo[NS], hhi[NS];
#pragma unroll
    for (int si = 1; si < NS; ++si) {
        hlo[si] = si == 1 ? 1 : a.stages[si - 1] + 1;
        hhi[si] = a.stages[si];
    }
    const int f0 = blockIdx.y * a.f_chunk;
    const int f1 = min(a.n_fund, f0 + a.f_chunk);
    if (top > 0) {
        int cnt = 0;
#pragma unroll 2
        for (int f = f0; f < f1; ++f) {
            const FundEntry *fe = a.fund + f;
            const int t = __ldg(&fe->t);
            const int st = min(__ldg(&fe->top_stage), top);
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int si = 1; si < NS; ++si) {
                if (si <= st) {
#pragma unroll
                    for (int h = 1; h <= JERK_MAX_HARMONIC; ++h) {
                        if (h >= hlo[si] && h <= hhi[si]) {
                            const float4 v = __ldg(reinterpret_cast<const float4 *>(
                                a.slots + __ldg(&fe->off[h - 1]) + p0));
                            s.x += v.x;
                            s.y += v.y;
                            s.z += v.z;
                            s.w += v.w;
                        }
                    }
                    const float sv[4] = {s.x, s.y, s.z, s.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (ok[si][c] && sv[c] > mx[si][c]) {
                            mx[si][c] = sv[c];
                            am[si][c] = t;
                        }
                        if (stats && ok[si][c]) {
                            c1[si] += sv[c];
                            c2[si] = fmaf(sv[c], sv[c], c2[si]);
                        }
                    }
                }
            }
            if (stats && ++cnt == 16) {
                cnt = 0;
#pragma unroll
                for (int si = 1; si < NS; ++si) {
                    d1[si] += (double)c1[si];
                    d2[si] += (double)c2[si];
                    c1[si] = c2[si] = 0.f;
                }
            }
        }
#pragma unroll
        for (int si = 1; si < NS; ++si) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (ok[si][c] && mx[si][c] >= 0.f) {
                    const unsigned long long packed =
                        ((unsigned long long)__float_as_uint(mx[si][c]) << 32) |
                        (unsigned long long)(0xFFFFFFFFu - (unsigned)am[si][c]);
                    if (gridDim.y == 1)
                        a.M[si][p0 + c] = packed;
                    else
                        atomicMax(a.M[si] + p0 + c, packed);
                }
            }
        }
    }
    if (stats) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int si = 1; si < NS; ++si) {
            double x1 = d1[si] + (double)c1[si], x2 = d2[si] + (double)c2[si];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x1 += __shfl_xor_sync(0xffffffffu, x1, o);
                x2 += __shfl_xor_sync(0xffffffffu, x2, o);
            }
            if (lane == 0) {
                red[si][0][warp] = x1;
                red[si][1][warp] = x2;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
            for (int si = 1; si < NS; ++si) {
                double s1 = 0.0, s2 = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    s1 += red[si][0][w];
                    s2 += red[si][1][w];
                }
                a.stat_part[(blk * a.n_stages + si) * 2] = s1;
                a.stat_part[(blk * a.n_stages + si) * 2 + 1] = s2;
            }
        }
    }
}

cudaError_t launch_harmonic(const HarmArgs &a, int64_t n_threads, int nblk_y, bool stats, cudaStream_t st) {
    const int64_t nblk = (n_threads + 255) / 256;
    dim3 grid((unsigned)nblk, (unsigned)nblk_y);
    switch (a.n_stages) {
        case 2: harmonic_kernel<2><<<grid, 256, 0, st>>>(a, stats); break;
        case 3: harmonic_kernel<3><<<grid, 256, 0, st>>>(a, stats); break;
        case 4: harmonic_kernel<4><<<grid, 256, 0, st>>>(a, stats); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Statistics (Sec. 3: mean and standard deviation) -> thresholds.  Partial
// sums are reduced in a fixed order, so the result is deterministic.
// ---------------------------------------------------------------------------
__global__ void finalise_stats_kernel(const double *part1, int64_t n1, const double *partH, int64_t nH,
                                      int n_stages, const double *counts, const float *thresh, int mode,
                                      double *stats_out, float *theta_out) {
    __shared__ double r1[256], r2[256];
    for (int si = 0; si < n_stages; ++si) {
        double s1 = 0.0, s2 = 0.0;
        if (mode == JERK_THRESH_SIGMA) {
            if (si == 0) {
                for (int64_t i = threadIdx.x; i < n1; i += blockDim.x) {
                    s1 += part1[2 * i];
                    s2 += part1[2 * i + 1];
                }
            } else {
                for (int64_t i = threadIdx.x; i < nH; i += blockDim.x) {
                    s1 += partH[(i * n_stages + si) * 2];
                    s2 += partH[(i * n_stages + si) * 2 + 1];
                }
            }
        }
        r1[threadIdx.x] = s1;
        r2[threadIdx.x] = s2;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                r1[threadIdx.x] += r1[threadIdx.x + o];
                r2[threadIdx.x] += r2[threadIdx.x + o];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double mu = 0.0, sd = 0.0;
            float theta = thresh[si];
            if (mode == JERK_THRESH_SIGMA && counts[si] > 0.0) {
                mu = r1[0] / counts[si];
                const double var = r2[0] / counts[si] - mu * mu;
                sd = sqrt(var > 0.0 ? var : 0.0);
                theta = (float)(mu + (double)thresh[si] * sd);
            }
            stats_out[2 * si] = mu;
            stats_out[2 * si + 1] = sd;
            theta_out[si] = theta;
        }
        __syncthreads();
    }
}

cudaError_t launch_finalise_stats(const double *part1, int64_t n1, const double *partH, int64_t nH,
                                  int n_stages, const double *counts, const float *thresh, int mode,
                                  double *stats_out, float *theta_out, cudaStream_t st) {
    finalise_stats_kernel<<<1, 256, 0, st>>>(part1, n1, partH, nH, n_stages, counts, thresh, mode, stats_out,
                                             theta_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Peak finding (Sec. 3: "peaks which are above some user specified
// threshold"; the 1-D rule is a reading): p is kept when
// M(p) > theta, M(p) > M(p-1) and M(p) >= M(p+1), a missing neighbour
// counting as -inf.  Kept cells are compacted with one atomic counter.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mval(unsigned long long x) { return __uint_as_float((unsigned)(x >> 32)); }

__global__ void peaks_kernel(PeakArgs a) {
    const int si = blockIdx.y;
    const int64_t n = a.n_cells[si];
    const unsigned long long *M = a.M[si];
    const float theta = a.theta[si];
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long x = M[p];
        const float v = mval(x);
        if (!(v > theta)) continue;
        const float l = p > 0 ? mval(M[p - 1]) : -FLT_MAX;
        const float r = p + 1 < n ? mval(M[p + 1]) : -FLT_MAX;
        if (v > l && v >= r) {
            const unsigned long long idx = atomicAdd(a.count, 1ull);
            if ((int64_t)idx < a.cap) {
                DevCand c;
                c.p = p;
                c.t = (int32_t)(0xFFFFFFFFu - (unsigned)(x & 0xFFFFFFFFull));
                c.stage_idx = si;
                c.power = v;
                c.item = a.item;
                a.out[idx] = c;
            }
        }
    }
}

cudaError_t launch_peaks(const PeakArgs &a, cudaStream_t st) {
    int64_t nmax = 0;
    for (int si = 0; si < a.n_stages; ++si) nmax = a.n_cells[si] > nmax ? a.n_cells[si] : nmax;
    int64_t nblk = (nmax + 255) / 256;
    if (nblk > 152 * 16) nblk = 152 * 16;
    if (nblk < 1) nblk = 1;
    dim3 grid((unsigned)nblk, (unsigned)a.n_stages);
    peaks_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Failure-path check: one thread waits, with the filter kernels' bounded
// wait, on a phase of an mbarrier that nothing completes; when the limit
// expires it sets the device error flag exactly as a filter CTA would, and
// returns.  Nothing else runs in the kernel.
// ---------------------------------------------------------------------------
__global__ void wait_check_kernel(int *err, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar, 1);
    if (!mbar_wait_for(&bar, 0, limit_ns)) atomicExch(err, 1);
}

cudaError_t launch_wait_check(int *err, uint64_t limit_ns, cudaStream_t st) {
    wait_check_kernel<<<1, 1, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Microbenchmarks for the roofline denominators that are not measured
// elsewhere: FP32 FMA throughput (8 independent FMA chains per thread, every
// SM full) and L2 read bandwidth (a buffer smaller than L2 read repeatedly
// with 16-byte loads).  Their outputs are consumed so nothing is elided.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) fma_peak_kernel(float *out, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // practically never
}

__global__ void __launch_bounds__(256) l2_read_kernel(const float4 *__restrict__ buf, int64_t n4, int reps,
                                                      float *out) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);                 // cached in L2 only
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    if (acc.x + acc.y + acc.z + acc.w == 12345.678f) out[threadIdx.x] = acc.x;
}

cudaError_t measure_peaks(int sms, double *fp32_tflops, double *l2_gbs) {
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *scratch = nullptr;
    float4 *buf = nullptr;
    const int64_t n4 = (64ll << 20) / 16;                    // 64 MB: inside the 129 MB L2
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&scratch, sizeof(float) * 512 * sms * 4);
    if (e == cudaSuccess) e = cudaMalloc(&buf, sizeof(float4) * n4);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(float4) * n4, st);
    float ms = 0.f;
    const int blocks = sms * 4, iters = 4096;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms up
        cudaEventRecord(e0, st);
        fma_peak_kernel<<<blocks, 512, 0, st>>>(scratch, iters, 0.999f, 1e-4f);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e == cudaSuccess)
        *fp32_tflops = 2.0 * 8 * 16 * (double)iters * blocks * 512 / (ms * 1e-3) / 1e12;
    const int reps = 20;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        l2_read_kernel<<<sms * 8, 256, 0, st>>>(buf, n4, reps, scratch);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e == cudaSuccess) *l2_gbs = (double)n4 * 16 * reps / (ms * 1e-3) / 1e9;
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(buf);
    cudaFree(scratch);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return e;
}

}  // namespace jerk
