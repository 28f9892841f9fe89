// Harmonic sums indexed by the highest harmonic (the sub-harmonic form).
//
// For a top harmonic at cell q of template t = (z, w):
//   S'_H(q, t) = sum_{h=1..H} P(round(h q / H), z_h, w_h),
// with (z_h, w_h) the grid point nearest to (h z / H, h w / H) and halves
// rounded away from zero.  Every template and every cell is a possible top
// harmonic, so the form needs the whole power plane; it serves banks whose
// plane fits on the device (the plane comes from jerk_plane).  Sec. 3 names
// the harmonic sum; this indexing is the one of the method's lineage (the
// fundamental-indexed sum of the main path adds the same terms where the
// rounding is exact).
//
// One thread per cell q walks the templates in ascending t, adds its H terms
// in h order in FP32, keeps the running (max, argmax) -- lowest t on equal
// sums -- and FP64 statistics partials; the plane is read through L2.
#include "jerk_internal.h"

namespace jerk {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int64_t round_ratio(int64_t a, int h, int H) {
    const int64_t m = (a < 0 ? -a : a) * h;
    const int64_t q = (2 * m + H) / (2 * H);
    return a < 0 ? -q : q;
}

struct SubArgs {
    const float *plane;          // [T][bN]
    int64_t bN;
    int32_t T, H, nz, zc, wc;    // zc = zmax / dz, wc = wmax / dw
    unsigned long long *M;       // [bN] packed max-projection
    double *part;                // [gridDim.x][2] statistics partials
};

__global__ void __launch_bounds__(kThreads) subharmonic_kernel(SubArgs a) {
    __shared__ double r1[kThreads / 32], r2[kThreads / 32];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < a.bN;
         q += (int64_t)gridDim.x * kThreads) {
        int64_t cell[JERK_MAX_HARMONIC];
#pragma unroll
        for (int h = 1; h <= JERK_MAX_HARMONIC; ++h)
            if (h <= a.H) cell[h - 1] = round_ratio(q, h, a.H);
        float best = -1.0f;
        int bt = 0;
        for (int t = 0; t < a.T; ++t) {
            const int zi = t % a.nz - a.zc, wi = t / a.nz - a.wc;
            float S = 0.0f;
            for (int h = 1; h <= a.H; ++h) {
                const int64_t th = (round_ratio(wi, h, a.H) + a.wc) * a.nz + (round_ratio(zi, h, a.H) + a.zc);
                S += __ldg(a.plane + th * a.bN + cell[h - 1]);
            }
            s1 += (double)S;
            s2 += (double)S * (double)S;
            if (S > best) {
                best = S;
                bt = t;
            }
        }
        a.M[q] = ((unsigned long long)__float_as_uint(best) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)bt);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = s1;
        r2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x1 = 0.0, x2 = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            x1 += r1[w];
            x2 += r2[w];
        }
        a.part[2 * blockIdx.x] = x1;
        a.part[2 * blockIdx.x + 1] = x2;
    }
}

// the partials in block order (deterministic) into sums[0..1]
__global__ void sum_partials_kernel(const double *part, int n, double *sums) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double x1 = 0.0, x2 = 0.0;
        for (int i = 0; i < n; ++i) {
            x1 += part[2 * i];
            x2 += part[2 * i + 1];
        }
        sums[0] = x1;
        sums[1] = x2;
    }
}

}  // namespace
}  // namespace jerk

extern "C" jerk_status jerk_subharmonic(jerk_plan pl, const float *d_plane, int64_t n, int32_t H,
                                        uint64_t *d_maxproj, double *d_sums, void *stream) {
    using namespace jerk;
    if (!pl || !d_plane || !d_maxproj || !d_sums || n < 1 || n > pl->prm.max_bins) return JERK_EINVAL;
    if (H < 1 || H > JERK_MAX_HARMONIC) return JERK_EINVAL;
    if (cudaSetDevice(pl->device) != cudaSuccess) return JERK_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamWaitEvent(st, pl->done, 0) != cudaSuccess) return JERK_ECUDA;
    SubArgs a;
    a.plane = d_plane;
    a.bN = (int64_t)pl->b * n;
    a.T = pl->T;
    a.H = H;
    a.nz = pl->nz;
    a.zc = pl->prm.zmax / pl->prm.dz;
    a.wc = pl->prm.wmax / pl->prm.dw;
    a.M = (unsigned long long *)d_maxproj;
    a.part = pl->d_stat_part;
    int64_t nblk = (a.bN + kThreads - 1) / kThreads;
    nblk = std::min<int64_t>(nblk, (int64_t)pl->sms * 8);
    nblk = std::min<int64_t>(nblk, pl->stat_part_cap / 2);
    if (nblk < 1) return JERK_ENOMEM;
    subharmonic_kernel<<<(unsigned)nblk, kThreads, 0, st>>>(a);
    sum_partials_kernel<<<1, 32, 0, st>>>(pl->d_stat_part, (int)nblk, d_sums);
    if (cudaGetLastError() != cudaSuccess) return JERK_ECUDA;
    if (cudaEventRecord(pl->done, st) != cudaSuccess) return JERK_ECUDA;
    return JERK_OK;
}
