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
// is the reading) and the stage-H max-projection over (z, w).  The harmonic
// rows P(h p, h z, h w) were written by the fused kernel into per-(h,
// fundamental) slots indexed by p (128-byte aligned).  A block covers
// HC_CELLS consecutive fundamental cells: HC_THREADS consumer threads own
// HC_PT cells each, and one producer warp streams the block's chunk of every
// row it needs (fundamentals in ascending t, h ascending) from HBM into a
// ring of HR shared-memory slots with bulk copies (cp.async.bulk +
// mbarrier), so HR x 8 KB are in flight per block whatever the consumers
// do.  The producer stages 32 table entries at a time in shared memory and
// one lane issues the copies, writing each slot's (t, top stage) beside it.
// Consumers sum their cells of each row in fixed h order (FP32), keep
// (max, argmax) per stage (lowest t on ties) and the statistics partials,
// and release each slot per warp.  Every wait is bounded (about one
// second); on expiry the block sets the error flag and leaves after its
// copies in flight have landed.
// ---------------------------------------------------------------------------
constexpr int HC_THREADS = 256;                 // consumer threads
constexpr int HC_PT = 8;                        // cells per consumer thread (two float4)
constexpr int HC_CELLS = HC_PT * HC_THREADS;    // fundamental cells per block
constexpr int HR = 11;                          // ring slots, one row chunk (HC_CELLS floats) each:
                                                // two blocks (ring + statics) fit an SM's shared memory

struct HarmEntry {                              // a table entry as the producer stages it
    int64_t off[JERK_MAX_HARMONIC];
    int t, st;
};

template <int NS>
__global__ void __launch_bounds__(HC_THREADS + 32, 2) harmonic_kernel(HarmArgs a, bool stats) {
    extern __shared__ __align__(128) float4 ring[];   // [HR][HC_CELLS / 4]
    __shared__ __align__(8) uint64_t full[HR];        // row chunk landed
    __shared__ __align__(8) uint64_t empty[HR];       // every consumer warp done with the slot
    __shared__ int2 meta[HR];                         // (t, top stage) of the slot's fundamental
    __shared__ HarmEntry tab[32];                     // the producer's current table entries
    __shared__ double red[JERK_MAX_STAGES][2][HC_THREADS / 32];
    __shared__ double dacc[NS - 1][2][HC_THREADS];    // per-thread FP64 statistics of stages 1.. (kept out of registers)
    constexpr int Q = HC_CELLS / 4;                   // float4 per slot
    const int tid = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * HC_CELLS;
    int topb = 0;   // highest stage index with cells in this block
#pragma unroll
    for (int si = 1; si < NS; ++si)
        if (c0 < a.n_cells[si]) topb = si;
    int hlo[NS], hhi[NS];
#pragma unroll
    for (int si = 1; si < NS; ++si) {
        hlo[si] = si == 1 ? 1 : a.stages[si - 1] + 1;
        hhi[si] = a.stages[si];
    }
    if (tid < HR) {
        mbar_init(&full[tid], 1);
        mbar_init(&empty[tid], HC_THREADS / 32);
    }
    __syncthreads();
    const int f0 = blockIdx.y * a.f_chunk;
    const int f1 = min(a.n_fund, f0 + a.f_chunk);

    if (tid >= HC_THREADS) {
        // ---- producer warp ----
        const int plane = tid - HC_THREADS;
        uint32_t bytes[NS];   // chunk bytes of a stage-si row: rows hold n_cells[si] cells, padded to 32
#pragma unroll
        for (int si = 1; si < NS; ++si) {
            const int64_t avail = ((a.n_cells[si] + 3) & ~(int64_t)3) - c0;
            bytes[si] = (uint32_t)(4 * (avail < HC_CELLS ? (avail > 0 ? avail : 0) : HC_CELLS));
        }
        int slot = 0, round = 0, issued = 0;
        bool good = topb > 0;
        for (int fb = f0; fb < f1 && good; fb += 32) {
            const int f = fb + plane;
            if (f < f1) {
                const FundEntry *fe = a.fund + f;
                const int st = min(__ldg(&fe->top_stage), topb);
                const int H = a.stages[st];
                tab[plane].t = __ldg(&fe->t);
                tab[plane].st = st;
#pragma unroll
                for (int h = 0; h < JERK_MAX_HARMONIC; ++h)
                    if (h < H) tab[plane].off[h] = __ldg(&fe->off[h]);
            }
            __syncwarp();
            if (plane == 0) {
                const int nb = min(32, f1 - fb);
                for (int k = 0; k < nb && good; ++k) {
                    const int t = tab[k].t, st = tab[k].st;
#pragma unroll
                    for (int si = 1; si < NS; ++si) {
                        if (si <= st) {
                            for (int h = hlo[si]; h <= hhi[si] && good; ++h) {
                                if (round > 0 && !mbar_wait_bounded(&empty[slot], (uint32_t)(round - 1) & 1u)) {
                                    good = false;
                                    break;
                                }
                                meta[slot] = make_int2(t, st);
                                const int64_t src = tab[k].off[h - 1] + c0;
                                // a skipped copy would leave the consumers waiting: give up
                                // (bounded) like an expired wait
                                if (!JERK_CHECK(src >= 0 && src + bytes[si] / 4 <= a.slot_cap, a.chk, kChkHarmCopy)) {
                                    good = false;
                                    break;
                                }
                                bulk_load(ring + slot * Q, a.slots + src, bytes[si], &full[slot]);
                                ++issued;
                                if (++slot == HR) {
                                    slot = 0;
                                    ++round;
                                }
                            }
                        }
                    }
                }
            }
            good = __shfl_sync(0xffffffffu, good, 0);
            __syncwarp();   // lane 0 done reading `tab`
        }
        if (plane == 0) {
            if (topb > 0 && !good) atomicExch(a.err, 1);
            // never leave with a copy still writing into this block's shared memory:
            // the last phase of each slot in use
            const int last = issued < HR ? issued : HR;
            for (int k = 0; k < last; ++k) {
                const int i = issued - 1 - k;
                mbar_wait_bounded(&full[i % HR], (uint32_t)(i / HR) & 1u);
            }
        }
    } else {
        // ---- consumers: thread tid owns cells p0 + 4u + c, u = 0..HC_PT/4-1 ----
        constexpr int U = HC_PT / 4;
        const int lane = tid & 31;
        const int64_t p0 = c0 + 4 * tid;
        float mx[NS][HC_PT];
        int am[NS][HC_PT];
        float c1[NS], c2[NS];
#pragma unroll
        for (int si = 0; si < NS; ++si) {
#pragma unroll
            for (int c = 0; c < HC_PT; ++c) {
                mx[si][c] = -1.0f;
                am[si][c] = 0;
            }
            if (si > 0) dacc[si - 1][0][tid] = dacc[si - 1][1][tid] = 0.0;
            c1[si] = c2[si] = 0.f;
        }
        // cell of (u, c): p0 + 4 HC_THREADS u + c
        auto cell_ok = [&](int si, int k) { return p0 + 4 * HC_THREADS * (k >> 2) + (k & 3) < a.n_cells[si]; };
        if (topb > 0) {
            int slot = 0, cnt = 0;
            uint32_t phase = 0;
            bool good = true;
            // every table entry has a top stage >= 1, so every fundamental has rows
            for (int f = f0; f < f1 && good; ++f) {
                // the fundamental's first row carries its (t, top stage)
                if (!mbar_wait_bounded(&full[slot], phase)) {
                    good = false;
                    break;
                }
                const int2 tm = meta[slot];
                const int t = tm.x, st = tm.y;
                float sv[HC_PT];
#pragma unroll
                for (int c = 0; c < HC_PT; ++c) sv[c] = 0.f;
#pragma unroll
                for (int si = 1; si < NS; ++si) {
                    if (si <= st && good) {
                        for (int h = hlo[si]; h <= hhi[si]; ++h) {
                            if (!mbar_wait_bounded(&full[slot], phase)) {
                                good = false;
                                break;
                            }
                            float4 v[U];
#pragma unroll
                            for (int u = 0; u < U; ++u) v[u] = ring[slot * Q + u * HC_THREADS + tid];
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&empty[slot]);
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                sv[4 * u] += v[u].x;
                                sv[4 * u + 1] += v[u].y;
                                sv[4 * u + 2] += v[u].z;
                                sv[4 * u + 3] += v[u].w;
                            }
                            if (++slot == HR) {
                                slot = 0;
                                phase ^= 1u;
                            }
                        }
                        if (!good) break;
#pragma unroll
                        for (int c = 0; c < HC_PT; ++c) {
                            const bool ok = cell_ok(si, c);
                            if (ok && sv[c] > mx[si][c]) {
                                mx[si][c] = sv[c];
                                am[si][c] = t;
                            }
                            if (stats && ok) {
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
                        dacc[si - 1][0][tid] += (double)c1[si];
                        dacc[si - 1][1][tid] += (double)c2[si];
                        c1[si] = c2[si] = 0.f;
                    }
                }
            }
            if (!good) {
                if (lane == 0) atomicExch(a.err, 1);
            } else {
#pragma unroll
                for (int si = 1; si < NS; ++si) {
#pragma unroll
                    for (int c = 0; c < HC_PT; ++c) {
                        if (cell_ok(si, c) && mx[si][c] >= 0.f) {
                            const int64_t p = p0 + 4 * HC_THREADS * (c >> 2) + (c & 3);
                            const unsigned long long packed =
                                ((unsigned long long)__float_as_uint(mx[si][c]) << 32) |
                                (unsigned long long)(0xFFFFFFFFu - (unsigned)am[si][c]);
                            if (!JERK_CHECK(p < a.n_cells[si], a.chk, kChkHarmStore)) continue;
                            if (gridDim.y == 1)
                                a.M[si][p] = packed;
                            else
                                atomicMax(a.M[si] + p, packed);
                        }
                    }
                }
            }
        }
        if (stats) {
            const int warp = tid >> 5;
#pragma unroll
            for (int si = 1; si < NS; ++si) {
                double x1 = dacc[si - 1][0][tid] + (double)c1[si], x2 = dacc[si - 1][1][tid] + (double)c2[si];
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
        }
    }
    __syncthreads();
    if (stats && tid == 0) {
        const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
        for (int si = 1; si < NS; ++si) {
            double s1 = 0.0, s2 = 0.0;
            for (int w = 0; w < HC_THREADS / 32; ++w) {
                s1 += red[si][0][w];
                s2 += red[si][1][w];
            }
            a.stat_part[(blk * a.n_stages + si) * 2] = s1;
            a.stat_part[(blk * a.n_stages + si) * 2 + 1] = s2;
        }
    }
}

template <int NS>
static cudaError_t launch_harmonic_ns(const HarmArgs &a, dim3 grid, bool stats, cudaStream_t st) {
    const int smem = HR * HC_CELLS * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(harmonic_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    harmonic_kernel<NS><<<grid, HC_THREADS + 32, smem, st>>>(a, stats);
    return cudaGetLastError();
}

int harmonic_cells_per_block() { return HC_CELLS; }

cudaError_t launch_harmonic(const HarmArgs &a, int nblk_y, bool stats, cudaStream_t st) {
    const int64_t nblk = (a.n_cells[1] + HC_CELLS - 1) / HC_CELLS;
    const dim3 grid((unsigned)nblk, (unsigned)nblk_y);
    switch (a.n_stages) {
        case 2: return launch_harmonic_ns<2>(a, grid, stats, st);
        case 3: return launch_harmonic_ns<3>(a, grid, stats, st);
        case 4: return launch_harmonic_ns<4>(a, grid, stats, st);
        default: return cudaErrorInvalidValue;
    }
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

cudaError_t launch_peaks(const PeakArgs &a, int sms, cudaStream_t st) {
    int64_t nmax = 0;
    for (int si = 0; si < a.n_stages; ++si) nmax = a.n_cells[si] > nmax ? a.n_cells[si] : nmax;
    int64_t nblk = (nmax + 255) / 256;
    if (nblk > (int64_t)sms * 16) nblk = (int64_t)sms * 16;
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

// the same FP32 work as packed FMAs (fma.rn.f32x2, two lanes per instruction):
// 8 independent chains of float2 per thread
__global__ void __launch_bounds__(512) fma2_peak_kernel(float *out, int iters, float a, float b) {
    float2 x[8];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = make_float2((float)(threadIdx.x + i) * 1e-3f, (float)i * 1e-3f);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i].x + x[i].y;
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

cudaError_t measure_packed_fma(int sms, double *tflops) {
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *scratch = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&scratch, sizeof(float) * 512 * sms * 4);
    float ms = 0.f;
    const int blocks = sms * 4, iters = 2048;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms up
        cudaEventRecord(e0, st);
        fma2_peak_kernel<<<blocks, 512, 0, st>>>(scratch, iters, 0.999f, 1e-4f);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    // 4 flops per packed FMA (two lanes, two flops each)
    if (e == cudaSuccess) *tflops = 4.0 * 8 * 16 * (double)iters * blocks * 512 / (ms * 1e-3) / 1e12;
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(scratch);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return e;
}

int device_sms(int device) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n < 1) return 1;
    return n;
}

int current_device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    return device_sms(dev);
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
