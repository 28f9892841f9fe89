// Fused overlap-and-save matched filtering (Sec. 2, Fig. 1): per CTA one
// segment of the spread spectrum and a group of templates.
//
//   1. forward FFT of the segment (once per CTA, kept in shared memory);
//   2. per template: pointwise multiply by the template spectrum (read from
//      the L2-resident group slice of the bank), inverse FFT in registers and
//      shared memory, drop the K-1 overlap, |.|^2;
//   3. epilogue in registers: running (max, argmax) per cell over the group
//      -> one packed 64-bit atomicMax per cell into the stage-1
//      max-projection; FP32/FP64 statistics (SIGMA mode); the harmonic rows
//      the harmonic sum needs are staged through shared memory and written
//      coalesced.  In plane mode the power rows are written instead.
//
// The power plane is never materialised in search mode.
#include "fft.cuh"
#include "jerk_internal.h"

namespace jerk {

// float swizzle for the staged power row (at most 2-way conflicts for the
// digit-reversed writes and 3-way for strided harmonic reads)
__device__ __forceinline__ int swzf(int a) { return a ^ ((a >> 5) & 31); }

template <int LOG2L, int MODE, bool STATS>
__global__ void __launch_bounds__(FftCfg<LOG2L>::NT)
conv_kernel(ConvArgs a) {
    using C = FftCfg<LOG2L>;
    constexpr int L = C::L, NT = C::NT;
    extern __shared__ float2 smem[];
    float2 *xs = smem;            // segment spectrum, swizzled
    float2 *work = smem + L;      // transposes / staged power row
    __shared__ double red[2][32];

    const int j = threadIdx.x;
    const int s = blockIdx.x;
    const int64_t seg0 = (int64_t)s * a.V;     // first output cell
    const int64_t in0 = seg0 - a.bM;           // first spread sample (even)

    // ---- 1. forward FFT of the spread segment -------------------------------
    float2 v[16];
    {
        FftTw<LOG2L, -1> twf;
        twf.init(j);
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int64_t q = in0 + j + NT * m;          // spread sample index
            float2 x = make_float2(0.f, 0.f);
            if (((q & 1) == 0) && q >= 0 && (q >> 1) < a.N) x = a.spec[q >> 1];
            v[m] = x;
        }
        fft_run<LOG2L, -1>(v, work, j, twf);
        const int rv = fft_rev<LOG2L>(j);
#pragma unroll
        for (int r = 0; r < 16; ++r) xs[swz(rv + NT * r)] = v[r];
    }
    __syncthreads();

    // ---- 2. templates of this group -----------------------------------------
    FftTw<LOG2L, +1> twi;
    twi.init(j);
    const int rv = fft_rev<LOG2L>(j);
    int64_t tb = (int64_t)a.t0 + (int64_t)blockIdx.y * a.tpg;
    int64_t te = tb + a.tpg;
    if (te > (int64_t)a.t0 + a.nt) te = (int64_t)a.t0 + a.nt;

    bool valid[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int cell = rv + NT * r;
        valid[r] = cell < a.V && seg0 + cell < a.bN;
    }
    float mx[16];
    int am[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        mx[r] = -1.0f;
        am[r] = 0;
    }
    double d1 = 0.0, d2 = 0.0;
    float c1 = 0.f, c2 = 0.f;
    int nchunk = 0;

    for (int64_t t = tb; t < te; ++t) {
        const float2 *ct = a.bank + t * L;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int f = j + NT * m;
            v[m] = cmul(xs[swz(f)], __ldg(ct + f));
        }
        fft_run<LOG2L, +1>(v, work, j, twi);
        float P[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) P[r] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);

        if constexpr (MODE == 0) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                if (valid[r] && P[r] > mx[r]) {
                    mx[r] = P[r];
                    am[r] = (int)t;
                }
            }
            if constexpr (STATS) {
                float s1 = 0.f, s2 = 0.f;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const float q = valid[r] ? P[r] : 0.f;
                    s1 += q;
                    s2 = fmaf(q, q, s2);
                }
                c1 += s1;
                c2 += s2;
                if (++nchunk == 8) {
                    d1 += (double)c1;
                    d2 += (double)c2;
                    c1 = c2 = 0.f;
                    nchunk = 0;
                }
            }
            const int e0 = __ldg(a.slot_beg + t), e1 = __ldg(a.slot_beg + t + 1);
            if (e0 < e1) {
                float *pw = reinterpret_cast<float *>(work);
                __syncthreads();                       // last pass reads of `work` done
#pragma unroll
                for (int r = 0; r < 16; ++r) pw[swzf(rv + NT * r)] = P[r];
                __syncthreads();
                for (int e = e0; e < e1; ++e) {
                    const int h = __ldg(a.slot_h + e);
                    const int64_t off = __ldg(a.slot_off + e);
                    const int64_t len = __ldg(a.slot_len + e);
                    // cells q = h p in [seg0, seg0 + V) with q < bN and p < len
                    const int64_t pf = (seg0 + h - 1) / h;
                    int64_t pl = (seg0 + a.V - 1) / h;
                    const int64_t pmax = (a.bN - 1) / h;
                    if (pl > pmax) pl = pmax;
                    if (pl > len - 1) pl = len - 1;
                    for (int64_t p = pf + j; p <= pl; p += NT)
                        a.slots[off + p] = pw[swzf((int)(h * p - seg0))];
                }
                // the next fft_run begins with a barrier before reusing `work`
            }
        } else {
            float *row = a.plane + (t - a.t0) * a.bN + seg0;
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (valid[r]) row[rv + NT * r] = P[r];
        }
    }

    if constexpr (MODE == 0) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (valid[r] && tb < te) {
                const unsigned long long packed =
                    ((unsigned long long)__float_as_uint(mx[r]) << 32) |
                    (unsigned long long)(0xFFFFFFFFu - (unsigned)am[r]);
                atomicMax(a.M1 + seg0 + rv + NT * r, packed);
            }
        }
        if constexpr (STATS) {
            d1 += (double)c1;
            d2 += (double)c2;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                d1 += __shfl_xor_sync(0xffffffffu, d1, o);
                d2 += __shfl_xor_sync(0xffffffffu, d2, o);
            }
            if ((j & 31) == 0) {
                red[0][j >> 5] = d1;
                red[1][j >> 5] = d2;
            }
            __syncthreads();
            if (j == 0) {
                double s1 = 0.0, s2 = 0.0;
                for (int w = 0; w < NT / 32; ++w) {
                    s1 += red[0][w];
                    s2 += red[1][w];
                }
                const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
                a.stat_part[2 * blk] = s1;
                a.stat_part[2 * blk + 1] = s2;
            }
        }
    }
}

size_t conv_smem_bytes(int log2L) { return (size_t)2 * ((size_t)1 << log2L) * sizeof(float2); }

template <int LOG2L, int MODE, bool STATS>
static cudaError_t launch_one(const ConvArgs &a, int ngroups, cudaStream_t st) {
    auto k = conv_kernel<LOG2L, MODE, STATS>;
    const size_t sm = conv_smem_bytes(LOG2L);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid(a.nseg, ngroups);
    k<<<grid, FftCfg<LOG2L>::NT, sm, st>>>(a);
    return cudaGetLastError();
}

template <int LOG2L>
static cudaError_t launch_L(int mode, bool stats, const ConvArgs &a, int ngroups, cudaStream_t st) {
    if (mode == 1) return launch_one<LOG2L, 1, false>(a, ngroups, st);
    if (stats) return launch_one<LOG2L, 0, true>(a, ngroups, st);
    return launch_one<LOG2L, 0, false>(a, ngroups, st);
}

cudaError_t launch_conv(int log2L, int mode, bool stats, const ConvArgs &a, int ngroups,
                        cudaStream_t st) {
    switch (log2L) {
        case 10: return launch_L<10>(mode, stats, a, ngroups, st);
        case 11: return launch_L<11>(mode, stats, a, ngroups, st);
        case 12: return launch_L<12>(mode, stats, a, ngroups, st);
        case 13: return launch_L<13>(mode, stats, a, ngroups, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jerk
