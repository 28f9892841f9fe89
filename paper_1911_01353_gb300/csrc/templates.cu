// FP64 template generation on the GPU (off the timed path).
//
// Sec. 2: "each filter fits a specific Fourier response for a given first
// frequency derivative z = fdot T^2 and second frequency derivative
// w = fddot T^3".  The response of a unit signal whose frequency,
// fdot T^2 and fddot T^3 at mid-observation are (r, z, w), at frequency
// offset q bins, is
//     rho(q; z, w) = int_{-1/2}^{1/2} exp(2 pi i (-q u + z u^2/2 + w u^3/6)) du
// and the matched-filter taps are c_d = conj(rho(d/b; z, w)), |d| <= b m(z, w).
//
// The integral is evaluated by composite 64-node Gauss-Legendre quadrature
// with at most 8 cycles of the integrand per panel (error far below FP64
// rounding).  Inner sums use the panel structure: with u = a_j + s_i,
//     rho(q) = sum_i exp(-2 pi i q s_i) sum_j c_{j,i} exp(-2 pi i q a_j),
// exp(-2 pi i q a_j) advanced by a complex recurrence over the uniform
// panel starts a_j, c_{j,i} = W_i (h/2) exp(2 pi i (z u^2/2 + w u^3/6)).
//
// The length-L spectrum of each tap vector is then taken by an FP64
// radix-2 FFT in shared memory and stored as FP32 with 1/L folded in (for
// the FP32 filter in the folded form described at template_fft_kernel).
#include <cmath>
#include <vector>

#include "jerk_internal.h"

namespace jerk {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute the derivative at the converged root
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

constexpr int kGL = 64;            // nodes per panel
constexpr double kCyclesPerPanel = 8.0;

__device__ __forceinline__ int halfwidth_dev(int z, int w, int pad) {
    return (4 * abs(z) + abs(w) + 7) / 8 + pad;
}

__global__ void taps_kernel(const int32_t *__restrict__ zt, const int32_t *__restrict__ wt,
                            const int32_t *__restrict__ tlist, int32_t t0, int b, int pad, int bM,
                            const double2 *__restrict__ gl, double2 *__restrict__ out) {
    extern __shared__ double2 chirp[];   // [panels * kGL]
    const int t = tlist ? tlist[blockIdx.x] : t0 + (int)blockIdx.x;
    const int K = 2 * bM + 1;
    double2 *dst = out + (int64_t)blockIdx.x * K;
    const int zi = zt[t], wi = wt[t];
    const double z = zi, w = wi;
    const int m = halfwidth_dev(zi, wi, pad);
    const double cyc = m + fabs(z) / 2.0 + fabs(w) / 8.0;     // max |d phase / du| in cycles
    const int panels = (int)ceil(cyc / kCyclesPerPanel) + 1;
    const double h = 1.0 / panels;
    const int nn = panels * kGL;
    for (int n = threadIdx.x; n < nn; n += blockDim.x) {
        const int jp = n / kGL, i = n % kGL;
        const double2 g = gl[i];
        const double u = -0.5 + h * (jp + 0.5 * (g.x + 1.0));
        double ph = z * u * u / 2.0 + w * u * u * u / 6.0;     // cycles
        ph -= rint(ph);
        double s, c;
        sincospi(2.0 * ph, &s, &c);
        const double wt_ = g.y * 0.5 * h;
        chirp[n] = make_double2(wt_ * c, wt_ * s);
    }
    __syncthreads();
    for (int d = -bM + (int)threadIdx.x; d <= bM; d += blockDim.x) {
        double2 res = make_double2(0.0, 0.0);
        if (abs(d) <= b * m) {
            const double q = (double)d / b;
            double rs, rc;
            sincospi(-2.0 * q * h, &rs, &rc);                  // ratio exp(-2 pi i q h)
            double es, ec;
            sincospi(q, &es, &ec);                             // exp(-2 pi i q (-1/2))
            double re = 0.0, im = 0.0;
            for (int i = 0; i < kGL; ++i) {
                const double si = 0.5 * h * (gl[i].x + 1.0);
                double ar = 0.0, ai = 0.0;
                double Er = ec, Ei = es;
                for (int jp = 0; jp < panels; ++jp) {
                    const double2 cv = chirp[jp * kGL + i];
                    ar = fma(cv.x, Er, fma(-cv.y, Ei, ar));
                    ai = fma(cv.x, Ei, fma(cv.y, Er, ai));
                    const double nr = Er * rc - Ei * rs;
                    const double ni = Er * rs + Ei * rc;
                    Er = nr;
                    Ei = ni;
                }
                double ps, pc;
                sincospi(-2.0 * q * si, &ps, &pc);
                re += ar * pc - ai * ps;
                im += ar * ps + ai * pc;
            }
            res = make_double2(re, -im);                       // c_d = conj(rho(d/b))
        }
        dst[d + bM] = res;
    }
}

// tw[i] = exp(+2 pi i i / L), i < L/2
__global__ void twiddle64_kernel(double2 *tw, int L) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L / 2) {
        double s, c;
        sincospi(2.0 * i / L, &s, &c);
        tw[i] = make_double2(c, s);
    }
}

// G[f] = (1/L) sum_{m<Kg} g[m] exp(+2 pi i f m / L): radix-2 DIT in shared
// memory.  Row i holds taps at index d + bM (bank-wide offset); the template's
// group uses offset bM - shift[i], i.e. g[m] = taps[i][m + shift[i]], m < klen[i].
//
// fold_r0 > 0 stores the row in the folded form the FP32 filter multiplies
// with (its inverse transform's first pass has radix R0 = fold_r0 over the
// elements f = j + (L/16)(i + (16/R0) k)): the spread segment has zeros at
// every odd cell, so its spectrum X has period L/2, and that pass splits
// into two DFTs of R0/2 points on, for f < L/2,
//   Ge[f] = G[f] + G[f + L/2],
//   Go[f] = (G[f] - G[f + L/2]) exp(+2 pi i k / R0),  k = (f / (L/16)) / (16 / R0),
// both computed in FP64 before the one rounding to FP32 and stored
// interleaved, row[2 f] = Ge[f], row[2 f + 1] = Go[f], so that one 16-byte
// shared-memory load gives a thread both factors of its spectrum value X[f].
// fold_r0 < 0 stores the paired form of the tensor-core filter (below); 0
// stores G as it is.
__global__ void template_fft_kernel(const double2 *__restrict__ taps, const int32_t *__restrict__ shift,
                                    const int32_t *__restrict__ klen, int K, int L, int log2L,
                                    const double2 *__restrict__ tw, int fold_r0, float2 *__restrict__ bank) {
    extern __shared__ double2 buf[];   // [L]
    const double2 *g = taps + (int64_t)blockIdx.x * K;
    const int sh = shift[blockIdx.x], kl = klen[blockIdx.x];
    for (int m = threadIdx.x; m < L; m += blockDim.x) {
        const int r = __brev(m) >> (32 - log2L);
        buf[r] = m < kl ? g[m + sh] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int len = 2; len <= L; len <<= 1) {
        const int half = len >> 1, step = L / len;
        for (int bfly = threadIdx.x; bfly < L / 2; bfly += blockDim.x) {
            const int grp = bfly / half, k = bfly % half;
            const int i0 = grp * len + k, i1 = i0 + half;
            const double2 wv = tw[k * step];
            const double2 x1 = buf[i1];
            const double2 v = make_double2(x1.x * wv.x - x1.y * wv.y, x1.x * wv.y + x1.y * wv.x);
            const double2 u = buf[i0];
            buf[i0] = make_double2(u.x + v.x, u.y + v.y);
            buf[i1] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
    float2 *dst = bank + (int64_t)blockIdx.x * L;
    const double inv = 1.0 / L;
    if (fold_r0 > 0) {
        const int half = L / 2, nt = L / 16, i0 = 16 / fold_r0;
        for (int f = threadIdx.x; f < L; f += blockDim.x) {
            double2 v;
            if (f < half) {
                v = make_double2(buf[f].x + buf[f + half].x, buf[f].y + buf[f + half].y);
            } else {
                const double2 d = make_double2(buf[f - half].x - buf[f].x, buf[f - half].y - buf[f].y);
                const int k = ((f - half) / nt) / i0;
                double sw, cw;
                sincospi(2.0 * k / fold_r0, &sw, &cw);
                v = make_double2(d.x * cw - d.y * sw, d.x * sw + d.y * cw);
            }
            const int slot = f < half ? 2 * f : 2 * (f - half) + 1;
            dst[slot] = make_float2((float)(v.x * inv), (float)(v.y * inv));
        }
        return;
    }
    if (fold_r0 < 0) {
        // paired form of the tensor-core filter: spectrum values f and f + P
        // (P = -fold_r0, bit log2 P of f clear) side by side as (Re f, Re f+P)
        // (Im f, Im f+P) at float2 slots 2 q and 2 q + 1, q = f with that bit
        // removed, so that one 16-byte load feeds a packed product of two
        // values
        const int P = -fold_r0;
        for (int q = threadIdx.x; q < L / 2; q += blockDim.x) {
            const int f = (q & (P - 1)) | ((q & ~(P - 1)) << 1);
            dst[2 * q] = make_float2((float)(buf[f].x * inv), (float)(buf[f + P].x * inv));
            dst[2 * q + 1] = make_float2((float)(buf[f].y * inv), (float)(buf[f + P].y * inv));
        }
        return;
    }
    for (int f = threadIdx.x; f < L; f += blockDim.x)
        dst[f] = make_float2((float)(buf[f].x * inv), (float)(buf[f].y * inv));
}

// out = max over the bank of max(|Re|, |Im|) (non-negative floats compare as ints)
__global__ void bank_maxabs_kernel(const float2 *__restrict__ bank, int64_t n, int *out) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = bank[i];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_int(m));
}

cudaError_t launch_bank_maxabs(const float2 *bank, int64_t n, float *out, int sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    bank_maxabs_kernel<<<sms * 4, 256, 0, st>>>(bank, n, reinterpret_cast<int *>(out));
    return cudaGetLastError();
}

cudaError_t launch_taps(const int32_t *zt, const int32_t *wt, const int32_t *tlist, int32_t t0, int32_t nt, int b,
                        int pad, int bM, const double2 *gl, int n_gl, double2 *out, cudaStream_t st) {
    if (n_gl != kGL) return cudaErrorInvalidValue;
    // shared memory sized for the widest template the bank can hold (half-width M = bM/b)
    const int M = bM / b;
    const int panels_max = (int)std::ceil((M + (M - pad) * 1.0) / kCyclesPerPanel) + 2;
    const size_t sm = (size_t)panels_max * kGL * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(taps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    taps_kernel<<<nt, 256, sm, st>>>(zt, wt, tlist, t0, b, pad, bM, gl, out);
    return cudaGetLastError();
}

cudaError_t launch_twiddles64(double2 *tw, int L, cudaStream_t st) {
    twiddle64_kernel<<<(L / 2 + 255) / 256, 256, 0, st>>>(tw, L);
    return cudaGetLastError();
}

cudaError_t launch_template_fft(const double2 *taps, const int32_t *shift, const int32_t *klen, int32_t nt, int K,
                                int L, const double2 *tw, int fold_r0, float2 *bank, cudaStream_t st) {
    int log2L = 0;
    while ((1 << log2L) < L) ++log2L;
    const size_t sm = (size_t)L * sizeof(double2);
    cudaError_t e =
        cudaFuncSetAttribute(template_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    template_fft_kernel<<<nt, 512, sm, st>>>(taps, shift, klen, K, L, log2L, tw, fold_r0, bank);
    return cudaGetLastError();
}

}  // namespace jerk
