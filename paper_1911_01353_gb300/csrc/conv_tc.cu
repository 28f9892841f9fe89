// Reduced-precision form of the fused overlap-and-save filter (Sec. 2,
// Fig. 1): the inverse transform of every (segment, template) product runs on
// the 5th-generation tensor cores as 64-point DFT blocks recast as dense
// products, with BF16 or FP16 operands and FP32 accumulation in tensor memory.
//
// Segment length L = 4096 = 64 x 64 (Cooley-Tukey, k = k1 + 64 k2 and
// n = 64 n1 + n2):
//   y[64 n1 + n2] = sum_k1 F[n1][k1] w^{k1 n2} sum_k2 Z[k1 + 64 k2] F[k2][n2],
// with F[a][b] = exp(+2 pi i a b / 64), w = exp(+2 pi i / L) and Z the
// product of the segment spectrum and the template spectrum (1/L folded into
// the bank).  One CTA holds two segments, so each step is a 128 x 128 x 128
// real product (complex values in real block form, [re | im]):
//   step 1: D1 = A1 B      A1[(seg, k1)][(re/im, k2)] = Z          (K-major)
//   twiddle U'[k1][n2] = D1 w^{k1 n2}   (FP32, in registers)
//   step 3: D3 = A3 B      A3[(seg, n2)][(re/im, k1)] = U'         (MN-major)
// where B is the real block form of F (the same matrix for both steps, F is
// symmetric).  D1 and D3 sit in tensor memory; every thread reads one row
// (tcgen05.ld), so the power |y|^2, the running max over the template group,
// the statistics and the harmonic rows are computed as in the FP32 kernel.
//
// Scaling: each segment spectrum is divided by max|X| * max|C| over the bank,
// so |Z| <= 1 and the FP16 operands of both steps stay in range (|U'| <= 64,
// |y| <= 4096 in FP32); powers are multiplied back before any use.
//
// One elected thread issues the MMAs (tcgen05.mma, operands in shared memory
// through matrix descriptors, no swizzle) and commits them to an mbarrier.
// Every wait on another agent (template bulk copies, MMA completion) is
// bounded (~1 s of %globaltimer); on expiry the CTA sets the plan's error flag
// (JERK_ETIMEOUT on the host), stops, drains its bulk copies and frees its
// tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "device_sync.cuh"
#include "fft.cuh"
#include "jerk_internal.h"

namespace jerk {
namespace {

constexpr int L = 4096, LOG2L = 12, NT = 256, SEGS = 2, THREADS = 512;
constexpr int WPAD = L + L / 16;                          // forward-transform work, per segment
constexpr uint32_t LBO = 128;                             // operand core-matrix stride along K (bytes)
constexpr uint32_t SBO = 2048;                            // ... along M / N (16 cores of 128 B along K)
constexpr int OPB = 128 * 128 * 2;                        // one 16-bit 128 x 128 operand
constexpr int OFF_A1 = 2 * L * 8;                         // after the two-deep template ring
constexpr int OFF_A3 = OFF_A1 + OPB;
constexpr int OFF_B = OFF_A3 + OPB;                       // B, then the twiddle table (one bulk copy)
constexpr int OFF_TW = OFF_B + OPB;                       // w^{k1 n2} for n2 = 2p, 2p + 1: float4 [p][k1] (re, re, im, im)
constexpr int OFF_AMX = OFF_TW + 64 * 64 * 8;             // uint16 [SEGS][L]: argmax offset in the group
constexpr int SMEM = OFF_AMX + SEGS * L * 2;              // 212 992 bytes
constexpr uint32_t TMEM_COLS = 256;                       // D1: columns 0..127, D3: 128..255
static_assert(SEGS * WPAD * 8 <= OFF_A3, "forward-transform work must fit below A3");

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    if constexpr (PREC == 1) {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

__device__ __forceinline__ void sts128(uint32_t addr, const uint32_t (&v)[8], int o) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[o]), "r"(v[o + 1]), "r"(v[o + 2]),
                 "r"(v[o + 3])
                 : "memory");
}

// shared-memory matrix descriptor: no swizzle, fixed version bits 46-48 = 0b001
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: D FP32, A/B BF16 (PREC 1) or FP16 (PREC 2),
// A K-major or MN-major, B K-major, M = N = 128
template <int PREC, bool A_MN>
__device__ __forceinline__ uint32_t idesc() {
    const uint32_t t = PREC == 1 ? 1u : 0u;
    return (1u << 4) | (t << 7) | (t << 10) | ((A_MN ? 1u : 0u) << 15) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
}

// D[128 x 128] (tensor memory) = A[128 x 128] B[128 x 128] as eight K = 16
// steps, issued by one elected lane of the calling warp: the whole warp
// executes it, so no lane diverges around the issue.  `ad` and `bd` are the
// step-0 shared-memory descriptors; step s starts 2 LBO bytes further along K,
// 16 more in the descriptors' 16-byte address field (which cannot carry:
// shared addresses are below 2^18).
static_assert((2 * LBO >> 4) == 16, "K-step increment of the descriptor address field");
template <int PREC, bool A_MN>
__device__ __forceinline__ void mma_tile_warp(uint32_t d_tmem, uint64_t ad, uint64_t bd) {
    asm volatile(
        "{\n\t.reg .pred e, f, t;\n\t.reg .b64 a, b;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 f, 0, 0;\n\t"
        "setp.eq.b32 t, 0, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, f;\n\t"
        "add.s64 a, %1, 16;\n\tadd.s64 b, %2, 16;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, t;\n\t"
        "add.s64 a, %1, 32;\n\tadd.s64 b, %2, 32;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, t;\n\t"
        "add.s64 a, %1, 48;\n\tadd.s64 b, %2, 48;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, t;\n\t"
        "add.s64 a, %1, 64;\n\tadd.s64 b, %2, 64;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, t;\n\t"
        "add.s64 a, %1, 80;\n\tadd.s64 b, %2, 80;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, t;\n\t"
        "add.s64 a, %1, 96;\n\tadd.s64 b, %2, 96;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, t;\n\t"
        "add.s64 a, %1, 112;\n\tadd.s64 b, %2, 112;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, t;\n\t}" ::"r"(d_tmem),
        "l"(ad), "l"(bd), "r"(idesc<PREC, A_MN>())
        : "memory");
}

// the elected lane's products so far arrive on `bar` when they complete
__device__ __forceinline__ void mma_commit_warp(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
            smem_u32(bar))
        : "memory");
}

// st.shared.u16 under a predicate, with no branch around it
__device__ __forceinline__ void st_shared_u16_if(bool pred, uint32_t addr, uint16_t v) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.shared.u16 [%1], %2;\n\t}" ::"r"((uint32_t)pred),
        "r"(addr), "h"(v)
        : "memory");
}

// acc0 += x0, acc1 += x1 in FP64.  A call, not inlined, so that it stays
// behind its branch (taken once in 32 templates): predicated in place, the
// slow FP64 conversions and adds would occupy the FP64 pipe every template.
__device__ __noinline__ void add_f64_pair(double *acc0, double *acc1, float x0, float x1) {
    *acc0 += (double)x0;
    *acc1 += (double)x1;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 2 x 16 consecutive FP32 columns of this thread's tensor-memory lane (at
// taddr0 and taddr1), both loads in flight before one wait; the wait carries
// the registers so that no use is scheduled before it
__device__ __forceinline__ void tmem_ld16x2(uint32_t taddr0, uint32_t taddr1, float (&x)[16], float (&y)[16]) {
    uint32_t r[16], q[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr0));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
          "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
        : "r"(taddr1));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(q[0]), "+r"(q[1]), "+r"(q[2]), "+r"(q[3]), "+r"(q[4]), "+r"(q[5]), "+r"(q[6]),
                   "+r"(q[7]), "+r"(q[8]), "+r"(q[9]), "+r"(q[10]), "+r"(q[11]), "+r"(q[12]), "+r"(q[13]),
                   "+r"(q[14]), "+r"(q[15])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        x[i] = __uint_as_float(r[i]);
        y[i] = __uint_as_float(q[i]);
    }
}

template <bool ROWS>
__device__ __forceinline__ int tc_bank_row(const ConvArgs &a, int k) {
    if constexpr (ROWS) return __ldg(a.rows + k);
    return k;
}

template <int PREC, int MODE, bool STATS, bool ROWS>
__global__ void __launch_bounds__(THREADS, 1) conv_tc_kernel(ConvArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float2 *ring = reinterpret_cast<float2 *>(sm);
    uint16_t *amx_s = reinterpret_cast<uint16_t *>(sm + OFF_AMX);
    __shared__ __align__(8) uint64_t full[2];                 // template bulk copy landed
    __shared__ __align__(8) uint64_t mbar1, mbar3, cbar;      // step 1 / step 3 done; constants landed
    __shared__ int issued[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int xmax_bits[SEGS];
    __shared__ double red[2][THREADS / 32];
    __shared__ double dacc[STATS ? 2 : 1][STATS ? THREADS : 1];
    __shared__ __align__(16) TplMeta tq[4];                 // (t, e0, e1) of template k at [k & 3]
    __shared__ __align__(16) RowEntries rent[2];            // slot entries of template k at [k & 1]

    const int tid = threadIdx.x;
    const int half = tid / NT, j = tid % NT;                  // forward-transform mapping
    const int warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, gcol = warp >> 2;           // tensor-memory lane quarter, column group
    const int row = 32 * quarter + lane;                      // operand / accumulator row: (seg, r)
    const int seg = row >> 6, r = row & 63;

    // (spectrum, template group) entry of this CTA: binary search of the CTA prefix
    int lo = 0, hi = a.n_work - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int)blockIdx.x >= __ldg(&a.grp[mid].cta0)) lo = mid; else hi = mid - 1;
    }
    const ItemDesc *itm = a.items + __ldg(&a.grp[lo].item);
    const int V = __ldg(&a.grp[lo].V), bM = __ldg(&a.grp[lo].bM);
    const int tb = __ldg(&a.grp[lo].tb), te = __ldg(&a.grp[lo].te);
    const int s_base = ((int)blockIdx.x - __ldg(&a.grp[lo].cta0)) * SEGS;
    const int64_t bN = itm->bN;

    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&mbar1, 1);
        mbar_init(&mbar3, 1);
        mbar_init(&cbar, 1);
        issued[0] = issued[1] = 0;
        xmax_bits[0] = xmax_bits[1] = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t tlane = (uint32_t)(32 * quarter) << 16;
    // B and the twiddle table: one bulk copy (not aliased by the transform work)
    if (tid == 0) bulk_load(sm + OFF_B, a.tc_const, (uint32_t)(OPB + 64 * 64 * 8), &cbar);

    // ---- 1. forward FFT of each spread segment (FP32) -------------------------
    {
        float2 v[16];
        float2 *work = reinterpret_cast<float2 *>(sm) + half * WPAD;
        const SyncNamed bar_half{1 + half, NT};
        FftTw<LOG2L, -1> twf;
        twf.init(j);
        const float2 *spec = itm->spec;
        const int64_t N = itm->N;
        const int64_t in0 = (int64_t)(s_base + half) * V - bM;   // first spread sample (even)
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int64_t q = in0 + j + NT * m;
            float2 x = make_float2(0.f, 0.f);
            if (((q & 1) == 0) && q >= 0 && (q >> 1) < N) x = spec[q >> 1];
            v[m] = x;
        }
        fft_pass0<LOG2L, -1>(v, twf);
        fft_store0<LOG2L>(v, work, j);
        fft_rest<LOG2L, -1>(v, work, j, twf, bar_half);
        const int rv = fft_rev<LOG2L>(j);
        bar_half();
#pragma unroll
        for (int m = 0; m < 16; ++m) work[rv + NT * m] = v[m];   // natural order
    }
    __syncthreads();
    // this thread's spectrum values in the tensor-core mapping: X[seg][r + 64 (16 gcol + i)]
    // Operand-build mapping: thread (ka, blk) forms Z for k = ka + 64 k2, k2 in
    // [8 blk, 8 blk + 8), of BOTH segments, so each template value is read from
    // shared memory once per CTA.  It keeps X[s][ka + 64 (8 blk + i)], s = 0, 1.
    // Values i and i + 1 are kept as packed pairs (xr: real parts, xi:
    // imaginary parts), matching the bank's paired form (f, f + 64).
    const int ka = tid & 63, blk = tid >> 6;
    float2 xr[SEGS][4], xi[SEGS][4];
    {
        float m[SEGS] = {0.f, 0.f};
#pragma unroll
        for (int s2 = 0; s2 < SEGS; ++s2) {
            const float2 *ws = reinterpret_cast<const float2 *>(sm) + s2 * WPAD;
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                const float2 x0 = ws[ka + 64 * (8 * blk + i)], x1 = ws[ka + 64 * (8 * blk + i + 1)];
                xr[s2][i >> 1] = make_float2(x0.x, x1.x);
                xi[s2][i >> 1] = make_float2(x0.y, x1.y);
                m[s2] = fmaxf(m[s2], fmaxf(fmaxf(fabsf(x0.x), fabsf(x0.y)), fmaxf(fabsf(x1.x), fabsf(x1.y))));
            }
        }
#pragma unroll
        for (int s2 = 0; s2 < SEGS; ++s2) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m[s2] = fmaxf(m[s2], __shfl_xor_sync(0xffffffffu, m[s2], o));
            if (lane == 0) atomicMax(&xmax_bits[s2], __float_as_int(m[s2]));   // non-negative: int order = float order
        }
    }
    if (tid == 64 && tb < te) {
        // the metadata pipeline's first stages: (t, e0, e1) of the first two
        // templates, t of the third, the slot entries of the first (later ones
        // are prefetched by cp.async in the loop)
        // (plane mode needs t only: it has no slot tables)
        for (int q = 0; q < 3 && tb + q < te; ++q) {
            const int t = __ldg(a.order + tb + q);
            const bool ent = MODE == 0 && q < 2;
            tq[(tb + q) & 3] = TplMeta{t, ent ? __ldg(a.slot_beg + t) : 0, ent ? __ldg(a.slot_beg + t + 1) : 0, 0};
        }
        if constexpr (MODE == 0) {
            const TplMeta m0 = tq[tb & 3];
            for (int i = 0; i < m0.e1 - m0.e0; ++i) {
                rent[tb & 1].h[i] = __ldg(a.slot_h + m0.e0 + i);
                rent[tb & 1].off[i] = __ldg(itm->slot_off + m0.e0 + i);
                rent[tb & 1].len[i] = __ldg(itm->slot_len + m0.e0 + i);
            }
        }
    }
    __syncthreads();                                          // the work buffers are free from here
    if (tid == 0)
        for (int b = 0; b < 2 && tb + b < te; ++b) {
            issued[b] = 1;
            bulk_load(ring + b * L, a.bank + (int64_t)tc_bank_row<ROWS>(a, tb + b) * L, (uint32_t)(L * sizeof(float2)),
                      &full[b]);
        }
    float psc;                                                // power = |y|^2 * psc (segment seg)
    {
        const float cm = __ldg(a.tc_cmax);
#pragma unroll
        for (int s2 = 0; s2 < SEGS; ++s2) {
            const float xm = __int_as_float(xmax_bits[s2]);
            const float sc = (xm > 0.f && cm > 0.f) ? 1.0f / (xm * cm) : 1.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                xr[s2][i] = make_float2(xr[s2][i].x * sc, xr[s2][i].y * sc);
                xi[s2][i] = make_float2(xi[s2][i].x * sc, xi[s2][i].y * sc);
            }
            if (s2 == seg) psc = 1.0f / (sc * sc);
        }
    }

    // cells of this thread: n = 64 (16 gcol + i) + r of segment seg.  n grows
    // with i, so the valid ones (n < V and within the spectrum) are the first
    // nvalid.
    const int seg0 = (s_base + seg) * V;
    int nvalid = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int n = 64 * (16 * gcol + i) + r;
        nvalid += (n < V && seg0 + n < bN) ? 1 : 0;
    }
    float mx[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) mx[i] = -1.0f;
    if constexpr (STATS) {
        dacc[0][tid] = 0.0;
        dacc[1][tid] = 0.0;
    }
    float c1 = 0.f, c2 = 0.f;
    // A1 rows 64 s + ka, K chunk blk (re) and 8 + blk (im)
    const uint32_t a1_r0 = smem_u32(sm + OFF_A1) + (ka >> 3) * SBO + (ka & 7) * 16 + blk * LBO;
    const uint32_t a1_r1 = a1_r0 + 8 * SBO;
    const uint32_t a3_col = smem_u32(sm + OFF_A3) + (r >> 3) * LBO + (r & 7) * 16 + (8 * seg + 2 * gcol) * SBO;
    const float4 *twt = reinterpret_cast<const float4 *>(sm + OFF_TW) + 8 * 64 * gcol + r;
    const uint32_t amx_t = smem_u32(amx_s + seg * L + 64 * 16 * gcol + r);   // this thread's cells, stride 128 B

    // ---- the three thread phases of one template --------------------------------
    // Warp 0 issues each product (one elected lane, so the warp never diverges
    // around an issue) right after the barrier that completes its operand.
    const uint64_t dA1 = sdesc(smem_u32(sm + OFF_A1)), dA3 = sdesc(smem_u32(sm + OFF_A3)),
                   dB = sdesc(smem_u32(sm + OFF_B));
    // A: Z = X C (scaled) -> A1 (K-major), from ring buffer `b`
    auto phase_a = [&](int b) {
        // template values f = ka + 64 (8 blk + i) and f + 64, paired in the bank
        const float4 *C = reinterpret_cast<const float4 *>(ring + b * L) + ka + 64 * 4 * blk;
        uint32_t pr[8], pi[8];                                // [seg 0: 0..3 | seg 1: 4..7]
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 c = C[64 * i];
            const float2 cr = make_float2(c.x, c.y), ci = make_float2(c.z, c.w);
#pragma unroll
            for (int s2 = 0; s2 < SEGS; ++s2) {
                // two complex products per packed instruction
                const float2 zr = sub2(mul2(xr[s2][i], cr), mul2(xi[s2][i], ci));
                const float2 zi = fma2(xr[s2][i], ci, mul2(xi[s2][i], cr));
                pr[4 * s2 + i] = pack2<PREC>(zr.x, zr.y);
                pi[4 * s2 + i] = pack2<PREC>(zi.x, zi.y);
            }
        }
        sts128(a1_r0, pr, 0);
        sts128(a1_r0 + 8 * LBO, pi, 0);
        sts128(a1_r1, pr, 4);
        sts128(a1_r1 + 8 * LBO, pi, 4);
    };
    // C: D1 -> twiddle -> A3 (MN-major)
    auto phase_c = [&]() {
        float ur[16], ui[16];
        tmem_ld16x2(tmem + tlane + 16 * gcol, tmem + tlane + 64 + 16 * gcol, ur, ui);
        uint32_t pr[8], pi[8];
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            // cells i, i + 1 at once: packed complex product with their twiddles
            const float4 w = twt[(i >> 1) * 64];
            const float2 re = make_float2(ur[i], ur[i + 1]), im = make_float2(ui[i], ui[i + 1]);
            const float2 wr = make_float2(w.x, w.y), wi = make_float2(w.z, w.w);
            const float2 ore = sub2(mul2(re, wr), mul2(im, wi));
            const float2 oim = fma2(re, wi, mul2(im, wr));
            pr[i >> 1] = pack2<PREC>(ore.x, ore.y);
            pi[i >> 1] = pack2<PREC>(oim.x, oim.y);
        }
        sts128(a3_col, pr, 0);
        sts128(a3_col + SBO, pr, 4);
        sts128(a3_col + 8 * LBO, pi, 0);
        sts128(a3_col + 8 * LBO + SBO, pi, 4);
    };
    // E: D3 -> power, running max, statistics, harmonic rows (search) or plane
    // rows.
    // The running max and the statistics use |y|^2 before the segment's power
    // scale psc (a monotone factor), applied when they leave the CTA.  The max
    // runs over all 16 cells: those past nvalid are never read back.  A warp
    // whose wait expired (`skip`) does none of it.
    auto phase_e = [&](int k, int it, bool skip) {
        if (skip) return;
        float yr[16], yi[16];
        tmem_ld16x2(tmem + tlane + 128 + 16 * gcol, tmem + tlane + 192 + 16 * gcol, yr, yi);
        float P[16];
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            const float2 re = make_float2(yr[i], yr[i + 1]), im = make_float2(yi[i], yi[i + 1]);
            const float2 p2 = fma2(re, re, mul2(im, im));    // two cells per packed instruction
            P[i] = p2.x;
            P[i + 1] = p2.y;
        }
        const int t = tq[k & 3].t;
        if constexpr (MODE == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                st_shared_u16_if(P[i] > mx[i], amx_t + 128 * i, (uint16_t)it);   // rare after the first templates
                mx[i] = fmaxf(mx[i], P[i]);
            }
            if constexpr (STATS) {
                // four independent chains over the thread's cells (two packed
                // pairs); cells outside the segment's valid range count as 0
                float2 a2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, q2[2] = {a2[0], a2[0]};
                if (nvalid == 16) {
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        const float2 p = make_float2(P[i], P[i + 1]);
                        a2[(i >> 1) & 1] = add2(a2[(i >> 1) & 1], p);
                        q2[(i >> 1) & 1] = fma2(p, p, q2[(i >> 1) & 1]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        const float2 p = make_float2(i < nvalid ? P[i] : 0.f, i + 1 < nvalid ? P[i + 1] : 0.f);
                        a2[(i >> 1) & 1] = add2(a2[(i >> 1) & 1], p);
                        q2[(i >> 1) & 1] = fma2(p, p, q2[(i >> 1) & 1]);
                    }
                }
                const float2 as = add2(a2[0], a2[1]), qs = add2(q2[0], q2[1]);
                c1 += as.x + as.y;
                c2 += qs.x + qs.y;
                if ((it & 31) == 31) {
                    // unscaled: the segment's scale is applied once, at the end
                    add_f64_pair(&dacc[0][tid], &dacc[1][tid], c1, c2);
                    c1 = c2 = 0.f;
                }
            }
            // harmonic rows: cell q = q0 + 64 i (q0 = seg0 + 1024 gcol + r) is
            // harmonic h of fundamental cell q / h when h | q; stored straight
            // from registers (lanes hold consecutive cells)
            const RowEntries &en = rent[k & 1];
            const int ne = tq[k & 3].e1 - tq[k & 3].e0;
            const int q0 = seg0 + 1024 * gcol + r;
            if (ne > 0) {
                // the rows hold scaled powers (P is not read again)
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const float2 ps = mul2(make_float2(P[i], P[i + 1]), make_float2(psc, psc));
                    P[i] = ps.x;
                    P[i + 1] = ps.y;
                }
            }
            for (int e = 0; e < ne; ++e) {
                const int h = en.h[e];
                float *dst = a.slots + en.off[e];
                const int len = (int)en.len[e];
                if ((h & (h - 1)) == 0) {
                    // h = 1, 2, 4, 8 divides 64: all of this thread's cells are
                    // harmonics of this h, or none is; cell i goes to row
                    // position quo + i dq (dq = 64 / h) while that is below len.
                    // The stride is a compile-time constant per h, so the 16
                    // stores take immediate offsets from one address.
                    const int lh = __ffs(h) - 1, ldq = 6 - lh;
                    if ((q0 & (h - 1)) == 0) {
                        const int quo = q0 >> lh;
                        const int iend = quo >= len ? 0 : min(nvalid, (len - quo + (1 << ldq) - 1) >> ldq);
                        float *d = dst + quo;
                        auto rows16 = [&](auto ldqc) {
                            constexpr int LDQ = decltype(ldqc)::value;
                            if (iend == 16) {
#pragma unroll
                                for (int i = 0; i < 16; ++i)
                                    if (JERK_CHECK(en.off[e] + quo + (i << LDQ) < a.slot_cap, a.chk, kChkTcRowStore))
                                        d[i << LDQ] = P[i];
                            } else {
#pragma unroll
                                for (int i = 0; i < 16; ++i)
                                    if (i < iend &&
                                        JERK_CHECK(en.off[e] + quo + (i << LDQ) < a.slot_cap, a.chk, kChkTcRowStore))
                                        d[i << LDQ] = P[i];
                            }
                        };
                        if (h == 1) rows16(std::integral_constant<int, 6>{});
                        else if (h == 2) rows16(std::integral_constant<int, 5>{});
                        else if (h == 4) rows16(std::integral_constant<int, 4>{});
                        else rows16(std::integral_constant<int, 3>{});
                    }
                } else {
                    // h = 3, 5, 6, 7: quotient and remainder stepped by 64 per cell
                    int quo = q0 / h, rem = q0 - quo * h;
                    const int dq = 64 / h, dr = 64 - dq * h;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        if (i < nvalid && rem == 0 && quo < len &&
                            JERK_CHECK(en.off[e] + quo < a.slot_cap, a.chk, kChkTcRowStore))
                            dst[quo] = P[i];
                        quo += dq;
                        rem += dr;
                        if (rem >= h) {
                            rem -= h;
                            quo += 1;
                        }
                    }
                }
            }
        } else {
            if (t >= a.t0 && t < a.t0 + a.nt) {
                const int64_t row0 = (int64_t)(t - a.t0) * bN + seg0;
                float *prow = a.plane + row0;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (i < nvalid &&
                        JERK_CHECK(row0 + 64 * (16 * gcol + i) + r < a.plane_len, a.chk, kChkTcPlaneStore))
                        prow[64 * (16 * gcol + i) + r] = P[i] * psc;
            }
        }
    };

    // ---- software pipeline over the group's templates ------------------------------
    // iteration it:  C(it) | A(it+1) with step 3 of it issued || E(it) with step 1
    // of it+1 issued, so each product runs while the threads work on the other.
    const int nt = te - tb;
    bool fail = !mbar_wait_bounded(&cbar, 0);
    fail = __any_sync(0xffffffffu, fail);
    if (nt > 0) {
        if (!fail) fail = !mbar_wait_bounded(&full[0], 0);
        fail = __any_sync(0xffffffffu, fail);
        if (!fail) phase_a(0);
        fence_async_smem();
        fail = __syncthreads_or(fail);
        if (!fail && warp == 0) {
            tc_fence_after();
            mma_tile_warp<PREC, false>(tmem, dA1, dB);
            mma_commit_warp(&mbar1);
        }
        if (!fail && tid == 32 && nt > 2) {                    // buffer 0 is read: template 2 next
            issued[0] += 1;
            bulk_load(ring, a.bank + (int64_t)tc_bank_row<ROWS>(a, tb + 2) * L, (uint32_t)(L * sizeof(float2)),
                      &full[0]);
        }
    }
    // `fail` is warp-uniform after each wait and CTA-uniform after each
    // __syncthreads_or; the loop is left only there, so every warp takes the
    // same barriers.
    for (int it = 0; it < nt; ++it) {
        // C(it): step 1 of template it has landed in D1
        if (!fail) fail = !mbar_wait_bounded(&mbar1, (uint32_t)it & 1u);
        fail = __any_sync(0xffffffffu, fail);
        tc_fence_after();
        if (!fail) phase_c();
        if (warp == 2) cp_async_wait_all();                   // the metadata issued last template
        tc_fence_before();
        fence_async_smem();
        if (__syncthreads_or(fail)) {
            fail = true;
            break;
        }
        if (warp == 2) {
            // Metadata pipeline (no L2-latency load between a product and the
            // epilogue that needs it): t of template k + 3, then (e0, e1) of
            // k + 2, then the slot entries of k + 1.  Every thread is past E of
            // the previous template, the last reader of the slots written here.
            const int k = tb + it;
            if (lane == 0) {
                if (k + 3 < te) cp_async<4>(&tq[(k + 3) & 3].t, a.order + k + 3);
                if (MODE == 0 && k + 2 < te) {
                    const int t2 = tq[(k + 2) & 3].t;
                    cp_async<4>(&tq[(k + 2) & 3].e0, a.slot_beg + t2);
                    cp_async<4>(&tq[(k + 2) & 3].e1, a.slot_beg + t2 + 1);
                }
            }
            if (MODE == 0 && k + 1 < te) {
                const TplMeta m1 = tq[(k + 1) & 3];
                if (lane < m1.e1 - m1.e0) {
                    const int e = m1.e0 + lane;
                    RowEntries &en = rent[(k + 1) & 1];
                    cp_async<4>(&en.h[lane], a.slot_h + e);
                    cp_async<8>(&en.off[lane], itm->slot_off + e);
                    cp_async<8>(&en.len[lane], itm->slot_len + e);
                }
            }
            cp_async_commit();
        }
        if (warp == 0) {
            // step 3 of template it (its operand A3 is complete)
            tc_fence_after();
            mma_tile_warp<PREC, true>(tmem + 128, dA3, dB);
            if (!inject_at(a, 3, it)) mma_commit_warp(&mbar3);
        }
        const bool more = it + 1 < nt;
        if (more) {
            // A(it + 1) while step 3 of template it runs
            const int b = (it + 1) & 1;
            fail = !mbar_wait_bounded(&full[b], (uint32_t)((it + 1) >> 1) & 1u);
            fail = __any_sync(0xffffffffu, fail);
            if (!fail) phase_a(b);
            fence_async_smem();
            if (__syncthreads_or(fail)) {
                fail = true;
                break;
            }
            if (tid == 32 && it + 3 < nt && !inject_at(a, 1, it + 3)) {   // buffer b is read: template it + 3 next
                issued[b] += 1;
                bulk_load(ring + b * L, a.bank + (int64_t)tc_bank_row<ROWS>(a, tb + it + 3) * L,
                          (uint32_t)(L * sizeof(float2)), &full[b]);
            }
            if (warp == 0) {
                // step 1 of template it + 1 (queued behind step 3 of it)
                tc_fence_after();
                mma_tile_warp<PREC, false>(tmem, dA1, dB);
                if (!inject_at(a, 2, it + 1)) mma_commit_warp(&mbar1);
            }
        }
        // E(it): step 3 of template it has landed in D3; step 1 of it + 1 runs meanwhile
        fail = !mbar_wait_bounded(&mbar3, (uint32_t)it & 1u);
        fail = __any_sync(0xffffffffu, fail);
        tc_fence_after();
        phase_e(tb + it, it, fail);
        tc_fence_before();
    }
    if (warp == 2) cp_async_wait_all();                       // no copy in flight past the loop
    fail = __syncthreads_or(fail);

    // ---- epilogue -----------------------------------------------------------------
    if (fail && tid == 0) atomicExch(a.err, 1);
    if constexpr (MODE == 0) {
        if (!fail && tb < te) {
            unsigned long long *M1 = itm->M1;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (i < nvalid) {
                    const int n = 64 * (16 * gcol + i) + r;
                    const int tw = __ldg(a.order + tb + amx_s[seg * L + n]);
                    const unsigned long long packed = ((unsigned long long)__float_as_uint(mx[i] * psc) << 32) |
                                                      (unsigned long long)(0xFFFFFFFFu - (unsigned)tw);
                    if (JERK_CHECK((int64_t)seg0 + n < bN, a.chk, kChkTcMaxProj)) atomicMax(M1 + seg0 + n, packed);
                }
            }
        }
        if constexpr (STATS) {
            double d1 = (dacc[0][tid] + (double)c1) * (double)psc;
            double d2 = (dacc[1][tid] + (double)c2) * ((double)psc * (double)psc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                d1 += __shfl_xor_sync(0xffffffffu, d1, o);
                d2 += __shfl_xor_sync(0xffffffffu, d2, o);
            }
            if (lane == 0) {
                red[0][warp] = d1;
                red[1][warp] = d2;
            }
            __syncthreads();
            if (tid == 0) {
                double s1 = 0.0, s2 = 0.0;
                for (int w = 0; w < THREADS / 32; ++w) {
                    s1 += red[0][w];
                    s2 += red[1][w];
                }
                a.stat_part[2 * (int64_t)blockIdx.x] = s1;
                a.stat_part[2 * (int64_t)blockIdx.x + 1] = s2;
            }
        }
    }
    if (tid == 0) {
        // never leave with a bulk copy still writing into this CTA's shared memory
        for (int b = 0; b < 2; ++b)
            if (issued[b] > 0) mbar_wait_bounded(&full[b], (uint32_t)(issued[b] - 1) & 1u);
        mbar_wait_bounded(&cbar, 0);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

template <int PREC, int MODE, bool STATS, bool ROWS>
cudaError_t launch_tc_one(const ConvArgs &a, int n_ctas, cudaStream_t st) {
    auto k = conv_tc_kernel<PREC, MODE, STATS, ROWS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    k<<<n_ctas, THREADS, SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_tc_prec(int mode, bool stats, const ConvArgs &a, int n_ctas, cudaStream_t st) {
    if (mode == 1) return launch_tc_one<PREC, 1, false, false>(a, n_ctas, st);
    if (a.rows) return stats ? launch_tc_one<PREC, 0, true, true>(a, n_ctas, st)
                             : launch_tc_one<PREC, 0, false, true>(a, n_ctas, st);
    return stats ? launch_tc_one<PREC, 0, true, false>(a, n_ctas, st)
                 : launch_tc_one<PREC, 0, false, false>(a, n_ctas, st);
}

}  // namespace

cudaError_t launch_conv_tc(int precision, int mode, bool stats, const ConvArgs &a, int n_ctas, cudaStream_t st) {
    if (!a.tc_const || !a.tc_cmax) return cudaErrorInvalidValue;
    if (precision == 1) return launch_tc_prec<1>(mode, stats, a, n_ctas, st);
    if (precision == 2) return launch_tc_prec<2>(mode, stats, a, n_ctas, st);
    return cudaErrorInvalidValue;
}

}  // namespace jerk
