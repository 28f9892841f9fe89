// Register/shared-memory FFT building blocks for the fused overlap-and-save
// kernel (the paper's "shared memory implementation of the FFT", Sec. 2,
// re-designed for sm_103a: 16 points per thread held in registers, radix-16
// butterflies in registers, padded shared-memory transposes between passes,
// no bank conflicts for any pass at L = 1024 .. 8192).
//
// Transform of length L = 2^LOG2L with NT = L/16 threads.  Each thread j
// enters with x[j + NT m], m = 0..15, in registers and leaves with
// y[rev(j) + NT r], r = 0..15, where y_v = sum_f x_f exp(SIGN 2 pi i f v / L)
// (unnormalised; SIGN = +1 inverse, -1 forward) and rev(j) is the
// mixed-radix digit reversal below.  Decimation in frequency, sub-problem-
// major storage: after pass s the data are A_s[rho][f] at logical index
// rho * N_s + f, physical index pad16(logical).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace jerk {

// Packed FP32 (add/sub/fma .f32x2, sm_100 and later) on the (re, im) pair of
// a complex value: one instruction where the scalar form takes two, with
// the same round-to-nearest result in each lane.  The packed forms run at the
// scalar FP32 rate but free an issue slot for the kernels' other
// instructions.  Host code (and device passes for older architectures, in
// host-side tests) takes the plain lane-by-lane form.
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
#define JERK_PACKED_F32 1
#else
#define JERK_PACKED_F32 0
#endif

__host__ __device__ __forceinline__ float2 add2(float2 a, float2 b) {
#if JERK_PACKED_F32
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 sub2(float2 a, float2 b) {
#if JERK_PACKED_F32
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 mul2(float2 a, float2 b) {
#if JERK_PACKED_F32
    return __fmul2_rn(a, b);
#else
    return make_float2(a.x * b.x, a.y * b.y);
#endif
}
// a * b + c, lane by lane
__host__ __device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
#if JERK_PACKED_F32
    return __ffma2_rn(a, b, c);
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}
// a * (k, k) + c
__host__ __device__ __forceinline__ float2 fma2k(float k, float2 a, float2 c) { return fma2(make_float2(k, k), a, c); }

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return add2(a, b); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return sub2(a, b); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a + SIGN i b and a - SIGN i b: the rotation swaps b's parts, so each lane
// takes its own scalar operation (no packed form without a register swap)
template <int SIGN>
__host__ __device__ __forceinline__ float2 cadd_i(float2 a, float2 b) {
    return SIGN > 0 ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, a.y - b.x);
}
template <int SIGN>
__host__ __device__ __forceinline__ float2 csub_i(float2 a, float2 b) {
    return cadd_i<-SIGN>(a, b);
}

// Padded shared-memory layout: one spare element after every 16, so that the
// strided transposes of every pass are free of bank conflicts and every
// address is a per-thread base plus a compile-time offset.
__device__ __forceinline__ int pad16(int a) { return a + (a >> 4); }

template <int LOG2L>
struct FftCfg {
    static constexpr int L = 1 << LOG2L;
    static constexpr int NT = L / 16;
    static constexpr int R0 = (LOG2L % 4) ? (1 << (LOG2L % 4)) : 16;   // radix of pass 0
    static constexpr int I0 = 16 / R0;                                  // pass-0 items per thread
    static constexpr int N0 = L / R0;                                   // sub-problem size after pass 0
    static constexpr int NP = (LOG2L % 4) ? LOG2L / 4 : LOG2L / 4 - 1;  // radix-16 passes after pass 0
    static_assert(LOG2L >= 10 && LOG2L <= 13, "L must be 1024..8192");
};

// ---------------------------------------------------------------------------
// Small DFTs in registers, natural order in and out.
// ---------------------------------------------------------------------------

template <int SIGN>
__host__ __device__ __forceinline__ float2 mul_i(float2 a) {  // (SIGN i) * a
    return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int SIGN>
__host__ __device__ __forceinline__ void dft2(float2 &a0, float2 &a1) {
    float2 s = cadd(a0, a1), d = csub(a0, a1);
    a0 = s;
    a1 = d;
}

template <int SIGN>
__host__ __device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
    const float2 s13 = cadd(a1, a3), e13 = csub(a1, a3);
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd_i<SIGN>(d02, e13);
    a3 = csub_i<SIGN>(d02, e13);
}

// exp(SIGN 2 pi i m / 16) as constants
template <int SIGN, int M>
__host__ __device__ __forceinline__ float2 w16() {
    constexpr float c[16] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                             0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                             -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                             0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
    constexpr float s[16] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                             1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                             0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                             -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f};
    return make_float2(c[M % 16], SIGN > 0 ? s[M % 16] : -s[M % 16]);
}

// The twiddles exp(SIGN 2 pi i m / 8) with m odd are c (+-1 +- i), c = 1/sqrt 2:
// a butterfly x0 +- w b with such a w is formed as x0 +- c (u, v), (u, v) the
// sums and differences of b's parts (eighth_root_parts), with fused
// multiply-adds: two scalar additions and two packed fused multiply-adds
// where a complex product and two complex additions take eight scalar
// instructions.  Complex additions without a rotation are one packed
// instruction; those with a +-i rotation (cadd_i) stay two scalar ones.
constexpr float kRsqrt2 = 0.70710678118654752f;

// (u, v) with w b = c (u, v) for w = exp(SIGN 2 pi i M / 8), M = 1 or 3
template <int SIGN, int M>
__host__ __device__ __forceinline__ float2 eighth_root_parts(float2 b) {
    static_assert(M == 1 || M == 3, "odd eighths of a turn below one half");
    // M = 1: w = c (1 + SIGN i);  M = 3: w = c (-1 + SIGN i)
    if constexpr (M == 1)
        return SIGN > 0 ? make_float2(b.x - b.y, b.y + b.x) : make_float2(b.x + b.y, b.y - b.x);
    else
        return SIGN > 0 ? make_float2(-b.x - b.y, b.x - b.y) : make_float2(b.y - b.x, -b.y - b.x);
}

// y_r = sum_k a_k exp(SIGN 2 pi i k r / 16): 4 x 4 split, k = k1 + 4 k2,
// r = r1 + 4 r2.  Layer 1: C[k1][r1] = DFT4 over k2; layer 2: for each r1, a
// DFT4 over k1 of C[k1][r1] w16^(k1 r1).  The twiddles w16^2 and w16^6 are
// formed inside their butterflies (eighth_root_parts), w16^4 = SIGN i is a swap.
template <int SIGN>
__host__ __device__ __forceinline__ void dft16(float2 (&a)[16]) {
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<SIGN>(a[k1], a[k1 + 4], a[k1 + 8], a[k1 + 12]);
    // a[k1 + 4 r1] = C[k1][r1]
    float2 y[16];
    // r1 = 0: no twiddles
    {
        float2 x0 = a[0], x1 = a[1], x2 = a[2], x3 = a[3];
        dft4<SIGN>(x0, x1, x2, x3);
        y[0] = x0;
        y[4] = x1;
        y[8] = x2;
        y[12] = x3;
    }
    // r1 = 1: x1 = C1 w^1, x2 = C2 w^2, x3 = C3 w^3
    {
        const float2 q = eighth_root_parts<SIGN, 1>(a[6]);         // w^2 C2 = c q
        const float2 s02 = fma2k(kRsqrt2, q, a[4]);
        const float2 d02 = fma2k(-kRsqrt2, q, a[4]);
        const float2 x1 = cmul(a[5], w16<SIGN, 1>()), x3 = cmul(a[7], w16<SIGN, 3>());
        const float2 s13 = cadd(x1, x3), e13 = csub(x1, x3);
        y[1] = cadd(s02, s13);
        y[9] = csub(s02, s13);
        y[5] = cadd_i<SIGN>(d02, e13);
        y[13] = csub_i<SIGN>(d02, e13);
    }
    // r1 = 2: x1 = C1 w^2, x2 = C2 w^4 = SIGN i C2, x3 = C3 w^6 = w^2 (SIGN i C3)
    {
        const float2 s02 = cadd_i<SIGN>(a[8], a[10]), d02 = csub_i<SIGN>(a[8], a[10]);
        const float2 e = cadd_i<SIGN>(a[9], a[11]), f = csub_i<SIGN>(a[9], a[11]);   // x1 + x3 = w^2 e, x1 - x3 = w^2 f
        const float2 qe = eighth_root_parts<SIGN, 1>(e);            // w^2 e = c qe
        const float2 qf = mul_i<SIGN>(eighth_root_parts<SIGN, 1>(f));   // SIGN i w^2 f = c qf (parts formed in place)
        y[2] = fma2k(kRsqrt2, qe, s02);
        y[10] = fma2k(-kRsqrt2, qe, s02);
        y[6] = fma2k(kRsqrt2, qf, d02);
        y[14] = fma2k(-kRsqrt2, qf, d02);
    }
    // r1 = 3: x1 = C1 w^3, x2 = C2 w^6, x3 = C3 w^9
    {
        const float2 q = eighth_root_parts<SIGN, 3>(a[14]);        // w^6 C2 = c q
        const float2 s02 = fma2k(kRsqrt2, q, a[12]);
        const float2 d02 = fma2k(-kRsqrt2, q, a[12]);
        const float2 x1 = cmul(a[13], w16<SIGN, 3>()), x3 = cmul(a[15], w16<SIGN, 9>());
        const float2 s13 = cadd(x1, x3), e13 = csub(x1, x3);
        y[3] = cadd(s02, s13);
        y[11] = csub(s02, s13);
        y[7] = cadd_i<SIGN>(d02, e13);
        y[15] = csub_i<SIGN>(d02, e13);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = y[i];
}

// y_r = sum_k a_k exp(SIGN 2 pi i k r / 8): k = k1 + 2 k2, r = r1 + 4 r2.
template <int SIGN>
__host__ __device__ __forceinline__ void dft8(float2 (&a)[8]) {
    dft4<SIGN>(a[0], a[2], a[4], a[6]);   // k1 = 0 -> C[0][r1] at a[2 r1]
    dft4<SIGN>(a[1], a[3], a[5], a[7]);   // k1 = 1 -> C[1][r1] at a[2 r1 + 1]
    // per r1: y[r1] = C0 + w8^r1 C1, y[r1 + 4] = C0 - w8^r1 C1
    float2 y[8];
    y[0] = cadd(a[0], a[1]);
    y[4] = csub(a[0], a[1]);
    {
        const float2 q = eighth_root_parts<SIGN, 1>(a[3]);          // w8^1 C1 = c q
        y[1] = fma2k(kRsqrt2, q, a[2]);
        y[5] = fma2k(-kRsqrt2, q, a[2]);
    }
    y[2] = cadd_i<SIGN>(a[4], a[5]);                                  // w8^2 = SIGN i
    y[6] = csub_i<SIGN>(a[4], a[5]);
    {
        const float2 q = eighth_root_parts<SIGN, 3>(a[7]);          // w8^3 C1 = c q
        y[3] = fma2k(kRsqrt2, q, a[6]);
        y[7] = fma2k(-kRsqrt2, q, a[6]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = y[i];
}

template <int SIGN, int R>
__host__ __device__ __forceinline__ void dft_small(float2 (&b)[R]) {
    if constexpr (R == 1) {
        // one point: its own transform
    } else if constexpr (R == 2) {
        dft2<SIGN>(b[0], b[1]);
    } else if constexpr (R == 4) {
        dft4<SIGN>(b[0], b[1], b[2], b[3]);
    } else if constexpr (R == 8) {
        dft8<SIGN>(b);
    } else {
        dft16<SIGN>(b);
    }
}

// b[r] *= w^r for r = 1..R-1 (running product)
template <int R>
__device__ __forceinline__ void twiddle(float2 *b, float2 w) {
    float2 acc = w;
    b[1] = cmul(b[1], acc);
#pragma unroll
    for (int r = 2; r < R; ++r) {
        acc = cmul(acc, w);
        b[r] = cmul(b[r], acc);
    }
}

// exp(SIGN 2 pi i num / den) for 0 <= num < den (den a power of two)
template <int SIGN>
__device__ __forceinline__ float2 unit_root(int num, int den) {
    float s, c;
    sincospif(2.0f * (float)num / (float)den, &s, &c);
    return make_float2(c, SIGN > 0 ? s : -s);
}

// Per-thread twiddle bases, constant across transforms; the factors of a
// pass are generated by a running product (registers only).
template <int LOG2L, int SIGN>
struct FftTw {
    using C = FftCfg<LOG2L>;
    float2 t0[C::I0];        // pass 0: w_L^{f1}, f1 = j + NT i
    float2 ts[C::NP];        // pass s (1..NP-1): w_{N_{s-1}}^{f'}, f' = j mod N_s
    __device__ __forceinline__ void init(int j) {
#pragma unroll
        for (int i = 0; i < C::I0; ++i) t0[i] = unit_root<SIGN>(j + C::NT * i, C::L);
        int nprev = C::N0;
#pragma unroll
        for (int s = 1; s <= C::NP; ++s) {
            const int ns = nprev / 16;
            ts[s - 1] = unit_root<SIGN>(j & (ns - 1), nprev);
            nprev = ns;
        }
    }
    template <int R>
    __device__ __forceinline__ void apply0(float2 *b, int i) const { twiddle<R>(b, t0[i]); }
    __device__ __forceinline__ void applys(float2 *a, int s) const { twiddle<16>(a, ts[s - 1]); }
};

// Twiddle factors read from tables in shared memory (built once per CTA by
// twiddle_tables below), for the inverse (SIGN = +1) or, conjugated, the
// forward transform.  Table 0: w_L^{f1 r} at [(r-1) * N0 + f1], or, when pass
// 0 has radix 16, in pairs (r, r + 1) for r = 1, 3, .., 15 as float4 [(r-1)/2]
// [f1] (one 16-byte load per two factors; the last pair's second half is
// padding); table s (1..NP-1): w_{N_{s-1}}^{f' r} in pairs (r, r + 1) as float4
// [(r-1)/2][f'] the same way.
template <int LOG2L, int SIGN>
struct FftTwSmem {
    using C = FftCfg<LOG2L>;
    const float2 *t0;
    const float2 *ts[C::NP > 1 ? C::NP - 1 : 1];
    int j;
    __device__ __forceinline__ static float2 cj(float2 w) { return SIGN > 0 ? w : make_float2(w.x, -w.y); }
    template <int R>
    __device__ __forceinline__ void apply0(float2 *b, int i) const {
        if constexpr (R == 16) {
            const float4 *p4 = reinterpret_cast<const float4 *>(t0) + j;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4 w = p4[k * C::N0];
                b[2 * k + 1] = cmul(b[2 * k + 1], cj(make_float2(w.x, w.y)));
                if (k < 7) b[2 * k + 2] = cmul(b[2 * k + 2], cj(make_float2(w.z, w.w)));
            }
        } else {
            const float2 *p = t0 + j + C::NT * i;
#pragma unroll
            for (int r = 1; r < R; ++r) b[r] = cmul(b[r], cj(p[(r - 1) * C::N0]));
        }
    }
    __device__ __forceinline__ void applys(float2 *a, int s) const {
        int ns = C::N0;
#pragma unroll
        for (int q = 0; q < s; ++q) ns /= 16;
        const float4 *p4 = reinterpret_cast<const float4 *>(ts[s - 1]) + (j & (ns - 1));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 w = p4[k * ns];
            a[2 * k + 1] = cmul(a[2 * k + 1], cj(make_float2(w.x, w.y)));
            if (k < 7) a[2 * k + 2] = cmul(a[2 * k + 2], cj(make_float2(w.z, w.w)));
        }
    }
};

// floats of shared memory the tables of FftTwSmem need
template <int LOG2L>
__host__ __device__ constexpr int twiddle_table_elems() {
    using C = FftCfg<LOG2L>;
    int n = C::R0 == 16 ? 16 * C::N0 : (C::R0 - 1) * C::N0;
    int ns = C::N0;
    for (int s = 1; s < C::NP; ++s) {
        ns /= 16;
        n += 16 * ns;
    }
    return n;
}

// fill the tables (inverse sign) with `nthr` cooperating threads
template <int LOG2L>
__device__ __forceinline__ void fill_twiddle_tables(float2 *tab, int tid, int nthr) {
    using C = FftCfg<LOG2L>;
    if constexpr (C::R0 == 16) {
        // pairs (r, r + 1), r = 1, 3, .., 15, as float4 [k][f1] (k = (r - 1) / 2); r = 16 is padding
        for (int e = tid; e < 16 * C::N0; e += nthr) {
            const int k = e / (2 * C::N0), rem = e % (2 * C::N0), f1 = rem >> 1, r = 2 * k + 1 + (rem & 1);
            tab[e] = r < 16 ? unit_root<+1>((f1 * r) & (C::L - 1), C::L) : make_float2(1.f, 0.f);
        }
    } else {
        for (int e = tid; e < (C::R0 - 1) * C::N0; e += nthr) {
            const int r = e / C::N0 + 1, f1 = e % C::N0;
            tab[e] = unit_root<+1>((f1 * r) & (C::L - 1), C::L);
        }
    }
    float2 *p = tab + (C::R0 == 16 ? 16 * C::N0 : (C::R0 - 1) * C::N0);
    int nprev = C::N0;
#pragma unroll
    for (int s = 1; s < C::NP; ++s) {
        const int ns = nprev / 16;
        for (int e = tid; e < 16 * ns; e += nthr) {
            const int k = e / (2 * ns), rem = e % (2 * ns), fp = rem >> 1, r = 2 * k + 1 + (rem & 1);
            p[e] = r < 16 ? unit_root<+1>((fp * r) & (nprev - 1), nprev) : make_float2(1.f, 0.f);
        }
        p += 16 * ns;
        nprev = ns;
    }
}

template <int LOG2L, int SIGN>
__device__ __forceinline__ FftTwSmem<LOG2L, SIGN> bind_twiddle_tables(const float2 *tab, int j) {
    using C = FftCfg<LOG2L>;
    FftTwSmem<LOG2L, SIGN> tw;
    tw.j = j;
    tw.t0 = tab;
    const float2 *p = tab + (C::R0 == 16 ? 16 * C::N0 : (C::R0 - 1) * C::N0);
    int ns = C::N0;
#pragma unroll
    for (int s = 1; s < C::NP; ++s) {
        ns /= 16;
        tw.ts[s - 1] = p;
        p += 16 * ns;
    }
    return tw;
}

// digit reversal: thread j's outputs sit at rev(j) + NT r
template <int LOG2L>
__device__ __forceinline__ int fft_rev(int j) {
    using C = FftCfg<LOG2L>;
    int t = j, acc = 0;
#pragma unroll
    for (int i = 0; i < C::NP - 1; ++i) {
        acc = acc * 16 + (t & 15);
        t >>= 4;
    }
    return acc * C::R0 + t;
}

// The transform, split so that a caller can interleave other work between
// pass 0 (registers only) and its shared-memory store.  `work` holds
// L + L/16 float2 (padded).  `Bar` is the barrier used between passes.
//
// pass 0: registers a[m] = x[j + NT m] -> a[i + I0 r] = pass-0 output r of item i
template <int LOG2L, int SIGN, class Tw>
__device__ __forceinline__ void fft_pass0(float2 (&a)[16], const Tw &tw) {
    using C = FftCfg<LOG2L>;
    constexpr int R0 = C::R0, I0 = C::I0;
#pragma unroll
    for (int i = 0; i < I0; ++i) {
        float2 b[R0];
#pragma unroll
        for (int k = 0; k < R0; ++k) b[k] = a[i + I0 * k];
        dft_small<SIGN, R0>(b);
        tw.template apply0<R0>(b, i);
#pragma unroll
        for (int r = 0; r < R0; ++r) a[i + I0 * r] = b[r];
    }
}

// Pass 0 of a transform whose input is a product X[f] G[f] with X of period
// L/2 (the spectrum of a segment with zeros at every odd sample), from the
// folded template of template_fft_kernel: a[m] for m < 8 holds X Ge (the sums
// G[f] + G[f + L/2]) and a[m + 8] holds X Go (the twiddled differences), f =
// j + NT m.  The radix-R0 DFT of each item then splits into two DFTs of R0/2
// points whose outputs are the even and the odd outputs of the full one:
// same results as fft_pass0 on the unfolded product, R0/2 fewer butterflies.
template <int LOG2L, int SIGN, class Tw>
__device__ __forceinline__ void fft_pass0_folded(float2 (&a)[16], const Tw &tw) {
    using C = FftCfg<LOG2L>;
    constexpr int R0 = C::R0, I0 = C::I0, RH = R0 / 2;
    static_assert(I0 * RH == 8, "the folded halves are a[0..7] and a[8..15]");
#pragma unroll
    for (int i = 0; i < I0; ++i) {
        float2 e[RH], o[RH];
#pragma unroll
        for (int k = 0; k < RH; ++k) {
            e[k] = a[i + I0 * k];
            o[k] = a[8 + i + I0 * k];
        }
        dft_small<SIGN, RH>(e);
        dft_small<SIGN, RH>(o);
        float2 b[R0];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            b[2 * r] = e[r];
            b[2 * r + 1] = o[r];
        }
        tw.template apply0<R0>(b, i);
#pragma unroll
        for (int r = 0; r < R0; ++r) a[i + I0 * r] = b[r];
    }
}

template <int LOG2L>
__device__ __forceinline__ void fft_store0(const float2 (&a)[16], float2 *__restrict__ work, int j) {
    using C = FftCfg<LOG2L>;
    constexpr int R0 = C::R0, I0 = C::I0, N0 = C::N0, NT = C::NT;
    float2 *w = work + pad16(j);
#pragma unroll
    for (int i = 0; i < I0; ++i)
#pragma unroll
        for (int r = 0; r < R0; ++r) w[((NT * i + r * N0) >> 4) * 17] = a[i + I0 * r];
}

// passes 1..NP; leaves y[rev(j) + NT r] in a[r]
//
// Pass s reads sub-problems of nprev = N0 / 16^(s-1) points, each handled by
// nprev / 16 consecutive threads, and (if not last) writes its outputs back
// into the same region.  So the hazards before a pass's loads (written by the
// previous pass's groups of 16 nprev / 16 = nprev threads) and before its
// stores (read by its own nprev / 16 threads) involve one warp only when
// those groups fit in a warp; there __syncwarp orders them and `bar` (the
// barrier over all threads of the transform) is not needed.  Pass 1's loads
// read what fft_store0 wrote across the whole transform: always `bar`.
template <int LOG2L, int SIGN, class Tw, class Bar>
__device__ __forceinline__ void fft_rest(float2 (&a)[16], float2 *__restrict__ work, int j, const Tw &tw,
                                         Bar bar) {
    using C = FftCfg<LOG2L>;
    int nprev = C::N0;
#pragma unroll
    for (int s = 1; s <= C::NP; ++s) {
        const int ns = nprev / 16;
        const int rho = j / ns, fp = j & (ns - 1);
        if (s > 1 && nprev <= 32)
            __syncwarp();
        else
            bar();
        {
            // loads in the order dft16's first radix-4 stage consumes them
            // (k1 + 4 k2, k2 fastest), so its butterflies start after four loads
            const float2 *r = work + pad16(rho * nprev + fp);
            const int step = ns + (ns >> 4);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
                for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = r[(k1 + 4 * k2) * step];
        }
        dft16<SIGN>(a);
        if (s < C::NP) {
            tw.applys(a, s);
            if (nprev <= 512)
                __syncwarp();
            else
                bar();
            float2 *w = work + pad16(rho * 16 * ns + fp);
            const int step = ns + (ns >> 4);
#pragma unroll
            for (int r = 0; r < 16; ++r) w[r * step] = a[r];
        }
        nprev = ns;
    }
}

struct SyncAll {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// named barrier over `n` threads (a multiple of 32)
struct SyncNamed {
    int id, n;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};

}  // namespace jerk
