// Matched-filter power at arbitrary points of the continuous (r, z, w)
// space: the response of Sec. 2 off the search grid, for refining candidates
// and for testing them against their 26 neighbours.
//
//   P(r, z, w) = |A|^2,  A = sum_k F_k conj(rho(k - r; z, w)),  |k - r| <= m(z, w),
//   rho(q; z, w) = int_{-1/2}^{1/2} exp(2 pi i (-q u + z u^2/2 + w u^3/6)) du,
//
// F the normalised spectrum (bins outside [0, N) zero), m(z, w) =
// ceil(|z|/2 + |w|/8) + P.  On the grid (r = p / b, integer z, w) this is the
// plane value P(p, z, w) the filter kernels compute.  Exchanging the sum and
// the integral, with the quadrature of the template bank (composite 64-node
// Gauss-Legendre, at most 8 cycles of the integrand per panel):
//   A = sum_n W_n (h/2) conj(e^{2 pi i phi(u_n)}) G(u_n),
//   phi(u) = z u^2/2 + w u^3/6,   G(u) = sum_k F_k e^{2 pi i (k - r) u}.
// One CTA per point: the spectrum window is staged in shared memory, threads
// split the nodes, G is summed in FP32 with the exponential advanced by a
// complex recurrence restarted exactly (FP64 phase) every 32 bins, and the
// node sums are reduced in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "jerk_internal.h"

namespace jerk {
namespace {

constexpr int kThreads = 256;
constexpr int kNodes = 64;                 // Gauss-Legendre nodes per panel (the bank's rule)
constexpr double kCyclesPerPanel = 8.0;
constexpr int kRestart = 32;               // bins between exact restarts of the recurrence
constexpr int kMaxWindow = 24000;          // bins staged per point (shared memory)

__device__ __host__ inline int halfwidth_at(double z, double w, int pad) {
    return (int)ceil(fabs(z) / 2.0 + fabs(w) / 8.0) + pad;
}

__global__ void __launch_bounds__(kThreads) power_at_kernel(const float2 *__restrict__ F, int64_t N,
                                                            const double *__restrict__ rzw, int pad,
                                                            const double2 *__restrict__ gl,
                                                            float *__restrict__ out) {
    extern __shared__ float2 win[];        // F[k0 .. k1]
    __shared__ double red[2][kThreads / 32];
    const double r = rzw[3 * blockIdx.x], z = rzw[3 * blockIdx.x + 1], w = rzw[3 * blockIdx.x + 2];
    const int m = halfwidth_at(z, w, pad);
    const int64_t k0 = max((int64_t)0, (int64_t)ceil(r - m));
    const int64_t k1 = min(N - 1, (int64_t)floor(r + m));
    const int nk = k1 >= k0 ? (int)(k1 - k0 + 1) : 0;
    for (int i = threadIdx.x; i < nk; i += blockDim.x) win[i] = F[k0 + i];
    __syncthreads();
    const double dk0 = (double)k0 - r;     // k - r of the first bin (|.| <= m + 1)
    const double cyc = m + fabs(z) / 2.0 + fabs(w) / 8.0;
    const int panels = (int)ceil(cyc / kCyclesPerPanel) + 1;
    const double h = 1.0 / panels;
    const int nn = panels * kNodes;
    double ar = 0.0, ai = 0.0;
    for (int n = threadIdx.x; n < nn; n += blockDim.x) {
        const int jp = n / kNodes, i = n - jp * kNodes;
        const double2 g = gl[i];
        const double u = -0.5 + h * (jp + 0.5 * (g.x + 1.0));
        double ph = z * u * u / 2.0 + w * u * u * u / 6.0;   // cycles
        ph -= rint(ph);
        double cs, cc;
        sincospi(2.0 * ph, &cs, &cc);
        const double wt = g.y * 0.5 * h;
        // e^{2 pi i u}: the per-bin ratio of the exponential
        float ss, sc;
        sincospif(2.0f * (float)u, &ss, &sc);
        float gr = 0.f, gi = 0.f;
        for (int kb = 0; kb < nk; kb += kRestart) {
            double p0 = (dk0 + kb) * u;
            p0 -= rint(p0);
            float es, ec;
            sincospif(2.0f * (float)p0, &es, &ec);
            const int ke = min(nk, kb + kRestart);
            for (int kk = kb; kk < ke; ++kk) {
                const float2 f = win[kk];
                gr = fmaf(f.x, ec, fmaf(-f.y, es, gr));
                gi = fmaf(f.x, es, fmaf(f.y, ec, gi));
                const float nr = ec * sc - es * ss;
                const float ni = ec * ss + es * sc;
                ec = nr;
                es = ni;
            }
        }
        ar += wt * (cc * (double)gr + cs * (double)gi);
        ai += wt * (cc * (double)gi - cs * (double)gr);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = ar;
        red[1][threadIdx.x >> 5] = ai;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sr = 0.0, si = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) {
            sr += red[0][i];
            si += red[1][i];
        }
        out[blockIdx.x] = (float)(sr * sr + si * si);
    }
}

}  // namespace
}  // namespace jerk

using namespace jerk;

namespace {

jerk_status from_cuda_r(cudaError_t e) {
    if (e == cudaSuccess) return JERK_OK;
    if (e == cudaErrorMemoryAllocation) return JERK_ENOMEM;
    return JERK_ECUDA;
}

#define RCHECK(x)                                      \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) return from_cuda_r(e_); \
    } while (0)

// normalise d_spec into the plan's workspace (after the plan's previous work)
jerk_status stage_spectrum(jerk_plan pl, const void *d_spec, int64_t n, cudaStream_t st, const float2 **out) {
    RCHECK(cudaStreamWaitEvent(st, pl->done, 0));
    if (pl->prm.norm_block > 0) {
        RCHECK(launch_normalise((const float2 *)d_spec, pl->d_spec_norm, n, pl->prm.norm_block, st));
        *out = pl->d_spec_norm;
    } else {
        *out = (const float2 *)d_spec;
    }
    return JERK_OK;
}

jerk_status power_at_host(jerk_plan pl, const float2 *F, int64_t n, const std::vector<double> &pts, float *h_out,
                          cudaStream_t st) {
    const int64_t count = (int64_t)pts.size() / 3;
    if (count == 0) return JERK_OK;
    int mmax = 0;
    for (int64_t i = 0; i < count; ++i) {
        const double z = pts[3 * i + 1], w = pts[3 * i + 2];
        if (!std::isfinite(pts[3 * i]) || !std::isfinite(z) || !std::isfinite(w)) return JERK_EINVAL;
        if (std::fabs(z) > 8192.0 || std::fabs(w) > 65536.0) return JERK_EINVAL;
        mmax = std::max(mmax, halfwidth_at(z, w, pl->prm.pad_bins));
    }
    const int win = 2 * mmax + 2;
    if (win > kMaxWindow) return JERK_EINVAL;
    const size_t smem = (size_t)win * sizeof(float2);
    double *d_pts = nullptr;
    float *d_out = nullptr;
    RCHECK(cudaMallocAsync((void **)&d_pts, sizeof(double) * pts.size(), st));
    cudaError_t e = cudaMallocAsync((void **)&d_out, sizeof(float) * count, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pts, pts.data(), sizeof(double) * pts.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(power_at_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int64_t b0 = 0; b0 < count && e == cudaSuccess; b0 += 65535) {
        const int nb = (int)std::min<int64_t>(65535, count - b0);
        power_at_kernel<<<nb, kThreads, smem, st>>>(F, n, d_pts + 3 * b0, pl->prm.pad_bins, pl->d_gl, d_out + b0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_out, sizeof(float) * count, cudaMemcpyDeviceToHost, st);
    if (d_pts) cudaFreeAsync(d_pts, st);
    if (d_out) cudaFreeAsync(d_out, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaEventRecord(pl->done, st);
    return from_cuda_r(e);
}

}  // namespace

extern "C" {

jerk_status jerk_power_at(jerk_plan pl, const void *d_spec, int64_t n, const double *h_rzw, int64_t count,
                          float *h_power, void *stream) {
    if (!pl || !d_spec || n < 1 || n > pl->prm.max_bins || count < 0 || (count > 0 && (!h_rzw || !h_power)))
        return JERK_EINVAL;
    if (!pl->share) return JERK_ESTATE;
    RCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    const float2 *F = nullptr;
    jerk_status s = stage_spectrum(pl, d_spec, n, st, &F);
    if (s != JERK_OK) return s;
    std::vector<double> pts(h_rzw, h_rzw + 3 * count);
    return power_at_host(pl, F, n, pts, h_power, st);
}

jerk_status jerk_refine(jerk_plan pl, const void *d_spec, int64_t n, const jerk_candidate *h_cands, int32_t count,
                        const double *h_step, const int32_t *h_half, jerk_refined *h_out, void *stream) {
    if (!pl || !d_spec || n < 1 || n > pl->prm.max_bins || count < 0 || !h_step || !h_half) return JERK_EINVAL;
    if (count > 0 && (!h_cands || !h_out)) return JERK_EINVAL;
    for (int i = 0; i < 3; ++i)
        if (h_half[i] < 0 || h_half[i] > 64 || !std::isfinite(h_step[i]) || h_step[i] < 0.0) return JERK_EINVAL;
    if (!pl->share) return JERK_ESTATE;
    RCHECK(cudaSetDevice(pl->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int nr = 2 * h_half[0] + 1, nzf = 2 * h_half[1] + 1, nwf = 2 * h_half[2] + 1;
    const int64_t G = (int64_t)nr * nzf * nwf;
    if ((int64_t)count * G > ((int64_t)1 << 26)) return JERK_EINVAL;
    std::vector<double> pts((size_t)(3 * count * G));
    for (int c = 0; c < count; ++c) {
        int64_t g = 0;
        for (int i = -h_half[0]; i <= h_half[0]; ++i)
            for (int j = -h_half[1]; j <= h_half[1]; ++j)
                for (int l = -h_half[2]; l <= h_half[2]; ++l, ++g) {
                    double *p = &pts[3 * ((size_t)c * G + g)];
                    p[0] = h_cands[c].r + i * h_step[0];
                    p[1] = (double)h_cands[c].z + j * h_step[1];
                    p[2] = (double)h_cands[c].w + l * h_step[2];
                }
    }
    const float2 *F = nullptr;
    jerk_status s = stage_spectrum(pl, d_spec, n, st, &F);
    if (s != JERK_OK) return s;
    std::vector<float> P((size_t)(count * G));
    s = power_at_host(pl, F, n, pts, P.data(), st);
    if (s != JERK_OK) return s;
    const int64_t centre = (G - 1) / 2;    // (i, j, l) = (0, 0, 0)
    for (int c = 0; c < count; ++c) {
        const float *pc = P.data() + (size_t)c * G;
        int64_t best = 0;
        for (int64_t g = 1; g < G; ++g)
            if (pc[g] > pc[best]) best = g;
        const double *p = &pts[3 * ((size_t)c * G + best)];
        jerk_refined &o = h_out[c];
        o.r = p[0];
        o.z = (float)p[1];
        o.w = (float)p[2];
        o.power = pc[best];
        o.power_in = pc[centre];
        o.is_peak = pc[centre] >= pc[best] ? 1 : 0;
        o.reserved = 0;
    }
    return JERK_OK;
}

}  // extern "C"
