// Fused overlap-and-save matched filtering (Sec. 2, Fig. 1).
//
// One CTA holds SEGS segments of the spread spectrum (one per group of NT
// threads) and walks a group of templates.  Templates are grouped by filter
// half-width, and each group uses its own overlap (tap offset bM) and hence
// its own segment length V = L - 2 bM, so short filters waste less of each
// transform on the overlap:
//   1. forward FFT of each segment (once per CTA, kept in shared memory);
//   2. per template: the template spectrum is staged into shared memory by a
//      TMA bulk copy (cp.async.bulk + mbarrier) issued during the previous
//      template's transform and shared by the SEGS segments; pointwise
//      multiply, inverse FFT in registers and padded shared memory, drop the
//      K-1 overlap, |.|^2.  The bank holds each template in a folded form
//      (sums and twiddled differences of its two spectrum halves): the
//      segment's spectrum repeats with period L/2, so the transform's first
//      pass splits into two half-size DFTs and each thread keeps only 8
//      spectrum values.  The butterflies act on the (re, im) pair of each
//      value with packed FP32 (fft.cuh); at L = 4096 the inverse transform's
//      twiddles come from tensor memory, where each thread keeps its own
//      (tmem.cuh), not from the shared-memory tables;
//   3. epilogue in registers: running (max, argmax) per cell over the group
//      -> one packed 64-bit atomicMax per cell into the stage-1
//      max-projection; statistics (SIGMA mode); the harmonic rows the
//      harmonic sum needs are staged through shared memory and written
//      coalesced.  In plane mode the power rows are written instead.
// Each template costs two barriers over its segment's threads; the metadata
// the epilogue and the row stores need (template index, slot-entry range and
// entries) is prefetched one template ahead into shared memory by cp.async,
// and the single-thread duties are spread over the segment's warps.
//
// The power plane is never materialised in search mode.  The only wait on
// another agent is the mbarrier of the bulk copy; it is bounded (about one
// second of %globaltimer) and on expiry the CTA records an error flag that
// the host reports as JERK_ETIMEOUT.
#include <type_traits>

#include "device_sync.cuh"
#include "fft.cuh"
#include "jerk_internal.h"
#include "rows.cuh"
#include "tmem.cuh"

namespace jerk {

template <int LOG2L>
struct ConvCfg {
    static constexpr int L = 1 << LOG2L;
    static constexpr int NT = L / 16;
    static constexpr int SEGS = LOG2L >= 13 ? 1 : 2;          // segments per CTA
    static constexpr int THREADS = SEGS * NT;
    static constexpr int MINB = THREADS >= 512 ? 1 : 512 / THREADS;
    static constexpr int WPAD = L + L / 16;                   // padded transpose buffer
    static constexpr bool TWS = LOG2L <= 12;                  // twiddles from shared-memory tables
    static constexpr int TWN = TWS ? twiddle_table_elems<LOG2L>() : 0;
    static constexpr int NBUF = LOG2L >= 13 ? 1 : 2;          // template buffers in flight
    // L = 4096: the inverse transform's twiddles in tensor memory, 64 columns
    // per thread (warps w, w + 4, .. share a lane range: 4 x 64 columns)
    static constexpr bool TMT = LOG2L == 12;
    static constexpr uint32_t TMCOLS = 256;
    // dynamic shared memory: NBUF x template | SEGS x work | twiddle tables |
    // SEGS x staged power row (float) | SEGS x argmax offset within the group (uint16)
    static constexpr size_t SMEM = sizeof(float2) * ((size_t)NBUF * L + (size_t)SEGS * WPAD + (size_t)TWN) +
                                   sizeof(float) * (size_t)SEGS * L + sizeof(uint16_t) * (size_t)SEGS * L;
};

template <int LOG2L, int SIGN>
__device__ __forceinline__ auto make_tw(const float2 *tab, int j) {
    if constexpr (ConvCfg<LOG2L>::TWS) {
        return bind_twiddle_tables<LOG2L, SIGN>(tab, j);
    } else {
        FftTw<LOG2L, SIGN> tw;
        tw.init(j);
        return tw;
    }
}

// The inverse transform's twiddles at L = 4096 read from tensor memory: this
// thread's 64 columns hold, at 0..31, the pass-0 factors w_L^{f1 r} for r =
// 1..15 in pairs (r, r + 1) as (re, im, re, im) (the last half padding), and
// at 32..63 the pass-1 factors w_256^{f' r} in the same form: the contents of
// this thread's entries of the shared-memory tables, copied once per CTA.
// Each pass reads them 8 columns at a time, the next 8 in flight while the
// current ones are used.
struct FftTwTmem {
    uint32_t ta;   // this thread's first column
    __device__ __forceinline__ static float2 w(const uint32_t (&r)[8], int q) {
        return make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
    }
    __device__ __forceinline__ static void run(uint32_t t, float2 *b) {
        uint32_t x[8], y[8];
        tmem_ld8(t, x);
        tmem_wait_ld8(x);
        tmem_ld8(t + 8, y);
#pragma unroll
        for (int q = 0; q < 4; ++q) b[1 + q] = cmul(b[1 + q], w(x, q));
        tmem_wait_ld8(y);
        tmem_ld8(t + 16, x);
#pragma unroll
        for (int q = 0; q < 4; ++q) b[5 + q] = cmul(b[5 + q], w(y, q));
        tmem_wait_ld8(x);
        tmem_ld8(t + 24, y);
#pragma unroll
        for (int q = 0; q < 4; ++q) b[9 + q] = cmul(b[9 + q], w(x, q));
        tmem_wait_ld8(y);
#pragma unroll
        for (int q = 0; q < 3; ++q) b[13 + q] = cmul(b[13 + q], w(y, q));
    }
    template <int R>
    __device__ __forceinline__ void apply0(float2 *b, int) const {
        static_assert(R == 16, "tensor-memory twiddles: L = 4096 only");
        run(ta, b);
    }
    __device__ __forceinline__ void applys(float2 *a, int) const { run(ta + 32, a); }
};

// Bank row (processing index) of position k of a work entry: the identity for
// whole-bank searches, a lookup when an item searches a sub-grid of the bank.
template <bool ROWS>
__device__ __forceinline__ int bank_row(const ConvArgs &a, int k) {
    if constexpr (ROWS) return __ldg(a.rows + k);
    return k;
}

template <int LOG2L, int MODE, bool STATS, bool ROWS>
__global__ void __launch_bounds__(ConvCfg<LOG2L>::THREADS, ConvCfg<LOG2L>::MINB)
conv_kernel(ConvArgs a) {
    using C = FftCfg<LOG2L>;
    using CC = ConvCfg<LOG2L>;
    constexpr int L = C::L, NT = C::NT, SEGS = CC::SEGS;
    constexpr int NBUF = CC::NBUF;
    extern __shared__ __align__(128) float2 smem[];
    __shared__ __align__(8) uint64_t full[NBUF];              // bulk copy of a template landed
    __shared__ int rel[NBUF];                                 // segments done reading a buffer
    __shared__ int issued[NBUF];                              // bulk copies issued per buffer
    __shared__ double red[2][32];
    __shared__ double dacc[STATS ? 2 : 1][STATS ? ConvCfg<LOG2L>::THREADS : 1];   // FP64 statistics per thread
    __shared__ __align__(16) TplMeta tq[SEGS][4];              // (t, e0, e1) of template k at [k & 3]
    __shared__ __align__(16) RowEntries rent[SEGS][2];         // slot entries of template k at [k & 1]

    const int tid = threadIdx.x;
    const int half = tid / NT;                                // which segment of the CTA
    const int j = tid - half * NT;
    float2 *work = smem + NBUF * L + half * CC::WPAD;         // transposes / staged power row
    float2 *twtab = smem + NBUF * L + SEGS * CC::WPAD;        // twiddle tables (TWS)
    float *stage = reinterpret_cast<float *>(twtab + CC::TWN) + half * L;   // power row awaiting slot stores
    uint16_t *amx = reinterpret_cast<uint16_t *>(reinterpret_cast<float *>(twtab + CC::TWN) + SEGS * L) +
                    half * L;                                  // argmax per cell, as t - tb
    __shared__ int sbound[SEGS][JERK_MAX_HARMONIC][2];        // per h: first and last p of the segment
    __shared__ const int64_t *srow[SEGS][2];                  // this segment's row offset / length tables
    __shared__ unsigned long long *sM1[SEGS];                 // this segment's stage-1 max-projection
    __shared__ uint32_t tslot;                                // tensor-memory base (CC::TMT)
    const SyncNamed bar_half{1 + half, NT};
    const int warp = tid >> 5;

    // (spectrum, template group) entry of this CTA: binary search of the CTA prefix
    int lo = 0, hi = a.n_work - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int)blockIdx.x >= __ldg(&a.grp[mid].cta0)) lo = mid; else hi = mid - 1;
    }
    const int g = lo;
    const int item = __ldg(&a.grp[g].item);
#define itm (a.items + item)
    const int V = __ldg(&a.grp[g].V), bM = __ldg(&a.grp[g].bM);
    const int tb = __ldg(&a.grp[g].tb), te = __ldg(&a.grp[g].te);
    const int s = ((int)blockIdx.x - __ldg(&a.grp[g].cta0)) * SEGS + half;
    const int seg0 = s * V;                                   // first output cell (< 2^31: max_bins <= 2^29)

    if (tid < NBUF) {
        mbar_init(&full[tid], 1);
        rel[tid] = 0;
        issued[tid] = 0;
    }
    if constexpr (CC::TWS) fill_twiddle_tables<LOG2L>(twtab, tid, CC::THREADS);
    if (j == 0) {
        srow[half][0] = itm->slot_off;
        srow[half][1] = itm->slot_len;
        sM1[half] = itm->M1;
    }
    if (j < JERK_MAX_HARMONIC) {
        // harmonic slots: cells q = h p in [seg0, seg0 + V), q < bN
        const int64_t bN = itm->bN;
        const int64_t h = j + 1;
        int64_t pl = (seg0 + V - 1) / h;
        const int64_t pmax = (bN - 1) / h;
        sbound[half][j][0] = (int)((seg0 + h - 1) / h);
        sbound[half][j][1] = (int)(pl < pmax ? pl : pmax);
    }
    if (j == 0 && tb < te) {
        // the metadata pipeline's first stages (later ones are prefetched in the loop)
        const int t0 = __ldg(a.order + tb);
        tq[half][tb & 3] = TplMeta{t0, __ldg(a.slot_beg + t0), __ldg(a.slot_beg + t0 + 1), 0};
        if (tb + 1 < te) tq[half][(tb + 1) & 3].t = __ldg(a.order + tb + 1);
    }
    if constexpr (CC::TMT)
        if (warp == 0) tmem_alloc_warp(smem_u32(&tslot), CC::TMCOLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (tid == 0)
        for (int b = 0; b < NBUF && tb + b < te; ++b) {
            issued[b] = 1;
            bulk_load(smem + b * L, a.bank + (int64_t)bank_row<ROWS>(a, tb + b) * L, (uint32_t)(L * sizeof(float2)),
                      &full[b]);
        }
    // this thread's columns: lanes 32 (warp % 4) + lane, columns 64 (warp / 4) ..
    const uint32_t tcol = CC::TMT ? tslot + ((uint32_t)(32 * (warp & 3)) << 16) + 64u * (uint32_t)(warp >> 2) : 0u;
    if constexpr (CC::TMT) {
        // copy this thread's entries of the inverse twiddle tables (pass 0: pairs
        // k = 0..7 at [k][j]; pass 1: pairs at [k][j mod 16]) into its columns
        const float4 *p0 = reinterpret_cast<const float4 *>(twtab) + j;
        const float4 *p1 = reinterpret_cast<const float4 *>(twtab + 16 * C::N0) + (j & 15);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float4 *src = c < 4 ? p0 + 2 * c * C::N0 : p1 + 2 * (c - 4) * 16;
            const int step = c < 4 ? C::N0 : 16;
            const float4 u = src[0], w = src[step];
            const float x[8] = {u.x, u.y, u.z, u.w, w.x, w.y, w.z, w.w};
            tmem_st8(tcol + 8 * c, x);
        }
        tmem_wait_st();
    }

    // ---- 1. forward FFT of the spread segment -------------------------------
    float2 v[16];
    {
        const auto twf = make_tw<LOG2L, -1>(twtab, j);
        const float2 *spec = itm->spec;
        const int64_t N = itm->N;
        const int64_t in0 = (int64_t)seg0 - bM;               // first spread sample (even)
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int64_t q = in0 + j + NT * m;               // spread sample index
            float2 x = make_float2(0.f, 0.f);
            if (((q & 1) == 0) && q >= 0 && (q >> 1) < N) x = spec[q >> 1];
            v[m] = x;
        }
        fft_pass0<LOG2L, -1>(v, twf);
        fft_store0<LOG2L>(v, work, j);
        fft_rest<LOG2L, -1>(v, work, j, twf, bar_half);
        const int rv = fft_rev<LOG2L>(j);
        bar_half();                                           // all reads of `work` done
#pragma unroll
        for (int r = 0; r < 16; ++r) work[rv + NT * r] = v[r];
        bar_half();
    }
    // each thread keeps the spectrum values it multiplies: X[j + NT m] for
    // m < 8 (the spread segment has zeros at its odd samples, so X has
    // period L/2 = 8 NT and X[j + NT (m + 8)] = X[j + NT m])
    float2 xr[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) xr[m] = work[j + NT * m];

    // ---- 2. templates of this group -----------------------------------------
    const auto twi = [&] {
        if constexpr (CC::TMT) return FftTwTmem{tcol};
        else return make_tw<LOG2L, +1>(twtab, j);
    }();
    const int rv = fft_rev<LOG2L>(j);
    unsigned vmask = 0;
    // Bit r of vmask: cell r of this thread is valid (within V and the
    // spectrum).  Bit 16: cells r < RSAFE of every thread of this segment are
    // valid (V >= NT RSAFE and the segment ends before bN), so the statistics
    // mask only r >= RSAFE; it is uniform over the segment, so over each warp.
    constexpr int RSAFE = 13;
    {
        const int64_t bN = itm->bN;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int cell = rv + NT * r;
            if (cell < V && seg0 + cell < bN) vmask |= 1u << r;
        }
        if (V >= NT * RSAFE && (int64_t)seg0 + NT * RSAFE <= bN) vmask |= 1u << 16;   // bit 16: the fast case
    }

    float mx[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) mx[r] = -1.0f;
    float fa0 = 0.f, fa1 = 0.f;                               // FP32 statistics partials (32 templates)
    if constexpr (STATS) {
        dacc[0][tid] = 0.0;
        dacc[1][tid] = 0.0;
    }
    // Template pipeline: template t sits in buffer b = (t - tb) % NBUF; the
    // last segment of the CTA to finish reading a buffer refills it with
    // template t + NBUF, so the segments never wait on each other.
    bool failed = false;
    // The last RD outputs r of every thread (cells rv + NT r >= NT (16 - RD))
    // lie in the overlap of every segment of this group, so the epilogue
    // skips them and the compiler drops the butterflies that only they need.
    // The loop is compiled for RD = 0, 1, 2 and the group's V picks one.
    auto template_loop = [&](auto rd) {
    constexpr int RK = 16 - decltype(rd)::value;              // outputs kept
    for (int k = tb; k < te; ++k) {                         // processing index
        const int it = k - tb;
        const int b = it % NBUF;
        const float2 *tsm = smem + b * L;
        // A thread whose wait expired reads a buffer that may still be landing;
        // its values are discarded: the whole segment leaves at the barrier below.
        const bool ok = mbar_wait_bounded(&full[b], (uint32_t)(it / NBUF) & 1u);
        // products with the folded template (sums for m < 8, twiddled
        // differences for m >= 8; stored interleaved, one 16-byte load gives
        // both factors of X[j + NT m]), then pass 0 as two half-size DFTs
        {
            const float4 *t4 = reinterpret_cast<const float4 *>(tsm);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const float4 g = t4[j + NT * m];
                v[m] = cmul(xr[m], make_float2(g.x, g.y));
                v[m + 8] = cmul(xr[m], make_float2(g.z, g.w));
            }
        }
        fft_pass0_folded<LOG2L, +1>(v, twi);
        // One barrier per template over the segment's threads: it reports an
        // expired wait, ends this segment's reads of the buffer, and orders the
        // previous template's reads of `work` and `stage` before their reuse.
        cp_async_wait_all();                                  // the copies issued last template
        if (named_any(1 + half, NT, !ok)) {
            if (j == 0) atomicExch(a.err, 1);
            failed = true;
            break;
        }
        // the segment's last warp releases (and, last of the segments, refills) the
        // buffer: the row stores' uneven last iteration falls on the first warps
        if (j == NT - 32) __threadfence_block();
        if (j == NT - 32 && atomicAdd(&rel[b], 1) == SEGS - 1) {
            rel[b] = 0;
            if (k + NBUF < te && !inject_at(a, 1, k + NBUF - tb)) {
                issued[b] += 1;
                bulk_load(smem + b * L, a.bank + (int64_t)bank_row<ROWS>(a, k + NBUF) * L, (uint32_t)(L * sizeof(float2)),
                          &full[b]);
            }
        }
        fft_store0<LOG2L>(v, work, j);
        // Metadata pipeline (L2-latency loads kept off the critical path, no
        // registers held): order[k + 2], then slot_beg of template k + 1, then the
        // slot entries of template k, each landing before the next template's
        // first barrier.  Issued here, where the pass-0 values are in shared memory.
        {
            // (on warps 1 and 2 -- warp 0 at L = 1024 -- away from the buffer release)
            if (j == 32) {
                if (k + 2 < te) cp_async<4>(&tq[half][(k + 2) & 3].t, a.order + k + 2);
                if (k + 1 < te) {
                    const int t1 = tq[half][(k + 1) & 3].t;
                    cp_async<4>(&tq[half][(k + 1) & 3].e0, a.slot_beg + t1);
                    cp_async<4>(&tq[half][(k + 1) & 3].e1, a.slot_beg + t1 + 1);
                }
            }
            if constexpr (MODE == 0) {
                const int ne = tq[half][k & 3].e1 - tq[half][k & 3].e0;   // this template's slot entries
                constexpr int EW = NT >= 128 ? 64 : 0;        // first thread of the entry copies
                const int i = j - EW;
                if (i >= 0 && i < ne) {
                    const int e = tq[half][k & 3].e0 + i;
                    RowEntries &en = rent[half][k & 1];
                    cp_async<4>(&en.h[i], a.slot_h + e);
                    cp_async<8>(&en.off[i], srow[half][0] + e);
                    cp_async<8>(&en.len[i], srow[half][1] + e);
                }
            }
            cp_async_commit();
        }
        if constexpr (MODE == 0)
            if (k > tb) {
                // the previous template's staged row
                const TplMeta mp = tq[half][(k - 1) & 3];
                if (mp.e0 < mp.e1)
                    store_rows(a, rent[half][(k - 1) & 1], mp.e1 - mp.e0, stage, sbound[half], (int)seg0, j, NT,
                               kChkRowStore);
            }
        fft_rest<LOG2L, +1>(v, work, j, twi, bar_half);
        float P[16];
#pragma unroll
        for (int r = 0; r < RK; ++r) P[r] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);

        if constexpr (MODE == 0) {
#pragma unroll
            for (int r = 0; r < RK; ++r) {
                if (P[r] > mx[r]) {
                    mx[r] = P[r];
                    amx[rv + NT * r] = (uint16_t)it;          // rare after the first templates
                }
            }
            if constexpr (STATS) {
                // invalid cells (overlap, beyond the spectrum) count as 0; the staged
                // row is never read back at those cells
                if (vmask >> 16) {
#pragma unroll
                    for (int r = RSAFE; r < RK; ++r) P[r] = (vmask >> r) & 1u ? P[r] : 0.f;
                } else {
#pragma unroll
                    for (int r = 0; r < RK; ++r) P[r] = (vmask >> r) & 1u ? P[r] : 0.f;
                }
                // four independent chains (two packed pairs of cells), then their sum
                float2 a2[2], q2[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const float2 p = make_float2(P[2 * i], P[2 * i + 1]);
                    a2[i] = p;
                    q2[i] = fma2(p, p, make_float2(0.f, 0.f));
                }
#pragma unroll
                for (int r = 4; r + 1 < RK; r += 2) {
                    const float2 p = make_float2(P[r], P[r + 1]);
                    a2[(r >> 1) & 1] = add2(a2[(r >> 1) & 1], p);
                    q2[(r >> 1) & 1] = fma2(p, p, q2[(r >> 1) & 1]);
                }
                if constexpr (RK & 1) {
                    a2[0].x += P[RK - 1];
                    q2[0].x = fmaf(P[RK - 1], P[RK - 1], q2[0].x);
                }
                const float2 as = add2(a2[0], a2[1]), qs = add2(q2[0], q2[1]);
                fa0 += as.x + as.y;
                fa1 += qs.x + qs.y;
                if ((it & 31) == 31) {
                    dacc[0][tid] += (double)fa0;
                    dacc[1][tid] += (double)fa1;
                    fa0 = fa1 = 0.f;
                }
            }
            // harmonic rows of this template: stage the power row now, store it
            // during the next template's transform (whose barriers order it)
            if (tq[half][k & 3].e0 < tq[half][k & 3].e1) {
#pragma unroll
                for (int r = 0; r < RK; ++r) {
                    // NT r only sets bits >= 8, which swzf neither reads nor changes
                    if constexpr (NT % 256 == 0)
                        stage[swzf(rv) + NT * r] = P[r];
                    else
                        stage[swzf(rv + NT * r)] = P[r];
                }
            }
        } else if (tq[half][k & 3].t >= a.t0 && tq[half][k & 3].t < a.t0 + a.nt) {
            const int t = tq[half][k & 3].t;
            const int64_t row0 = (int64_t)(t - a.t0) * (2 * (int64_t)a.items[0].N) + seg0;
            float *row = a.plane + row0;
#pragma unroll
            for (int r = 0; r < RK; ++r)
                if (((vmask >> r) & 1u) && JERK_CHECK(row0 + rv + NT * r < a.plane_len, a.chk, kChkPlaneStore))
                    row[rv + NT * r] = P[r];
        }
    }
    };
    if constexpr (LOG2L <= 12) {
        // (at L = 8192 the three copies spill)
        const int rd = MODE == 0 ? 16 - (V + NT - 1) / NT : 0;
        if (rd >= 2)
            template_loop(std::integral_constant<int, 2>{});
        else if (rd == 1)
            template_loop(std::integral_constant<int, 1>{});
        else
            template_loop(std::integral_constant<int, 0>{});
    } else {
        template_loop(std::integral_constant<int, 0>{});
    }

    cp_async_wait_all();
    if constexpr (MODE == 0) {
        bar_half();
        if (!failed && te > tb) {
            const TplMeta mp = tq[half][(te - 1) & 3];
            if (mp.e0 < mp.e1)
                store_rows(a, rent[half][(te - 1) & 1], mp.e1 - mp.e0, stage, sbound[half], (int)seg0, j, NT,
                           kChkRowStore);
        }
    }
    tmem_fence_before();
    __syncthreads();
    if constexpr (CC::TMT)
        if (warp == 0) {
            tmem_fence_after();
            tmem_dealloc_warp(tslot, CC::TMCOLS);
        }
    if (tid == 0) {
        // never leave with a bulk copy still writing into this CTA's shared memory
        for (int b = 0; b < NBUF; ++b)
            if (issued[b] > 0) mbar_wait_bounded(&full[b], (uint32_t)(issued[b] - 1) & 1u);
    }
    if constexpr (MODE == 0) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (((vmask >> r) & 1u) && tb < te && !failed) {
                const unsigned long long packed =
                    ((unsigned long long)__float_as_uint(mx[r]) << 32) |
                    (unsigned long long)(0xFFFFFFFFu - (unsigned)__ldg(a.order + tb + amx[rv + NT * r]));
                if (JERK_CHECK((int64_t)seg0 + rv + NT * r < itm->bN, a.chk, kChkMaxProj))
                    atomicMax(sM1[half] + seg0 + rv + NT * r, packed);
            }
        }
        if constexpr (STATS) {
            double d1 = dacc[0][tid] + (double)fa0;
            double d2 = dacc[1][tid] + (double)fa1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                d1 += __shfl_xor_sync(0xffffffffu, d1, o);
                d2 += __shfl_xor_sync(0xffffffffu, d2, o);
            }
            if ((tid & 31) == 0) {
                red[0][tid >> 5] = d1;
                red[1][tid >> 5] = d2;
            }
            __syncthreads();
            if (tid == 0) {
                double s1 = 0.0, s2 = 0.0;
                for (int w = 0; w < CC::THREADS / 32; ++w) {
                    s1 += red[0][w];
                    s2 += red[1][w];
                }
                const int64_t blk = blockIdx.x;
                a.stat_part[2 * blk] = s1;
                a.stat_part[2 * blk + 1] = s2;
            }
        }
    }
}

#undef itm

int conv_segs_per_cta(int log2L) { return log2L >= 13 ? 1 : 2; }

int conv_fold_radix(int log2L) { return (log2L % 4) ? (1 << (log2L % 4)) : 16; }

template <int LOG2L, int MODE, bool STATS, bool ROWS = false>
static cudaError_t launch_one(const ConvArgs &a, int n_ctas, cudaStream_t st) {
    using CC = ConvCfg<LOG2L>;
    auto k = conv_kernel<LOG2L, MODE, STATS, ROWS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::SMEM);
    if (e != cudaSuccess) return e;
    k<<<n_ctas, CC::THREADS, CC::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int LOG2L>
static cudaError_t launch_L(int mode, bool stats, const ConvArgs &a, int n_ctas, cudaStream_t st) {
    if (mode == 1) return launch_one<LOG2L, 1, false>(a, n_ctas, st);
    if (a.rows) return stats ? launch_one<LOG2L, 0, true, true>(a, n_ctas, st)
                             : launch_one<LOG2L, 0, false, true>(a, n_ctas, st);
    if (stats) return launch_one<LOG2L, 0, true>(a, n_ctas, st);
    return launch_one<LOG2L, 0, false>(a, n_ctas, st);
}

cudaError_t launch_conv(int log2L, int mode, bool stats, const ConvArgs &a, int n_ctas, cudaStream_t st) {
    switch (log2L) {
        case 10: return launch_L<10>(mode, stats, a, n_ctas, st);
        case 11: return launch_L<11>(mode, stats, a, n_ctas, st);
        case 12: return launch_L<12>(mode, stats, a, n_ctas, st);
        case 13: return launch_L<13>(mode, stats, a, n_ctas, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jerk
