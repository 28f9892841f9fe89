// Candidate extraction that allocates nothing.
//
// Some callers cannot allocate device memory when they want candidates: a
// real-time pipeline stage that reserved all of its memory before observing
// started (a cudaMalloc there can synchronise the device and stall for
// milliseconds), or a host program whose device memory is owned by another
// allocator, such as a framework's caching allocator, that the library must
// not bypass.  jerk_peaks_noalloc serves them: it is a variant of the
// library's peak-finding kernel whose scratch memory (per-block counts,
// turned into output offsets) is a fixed array in this file rather than a
// buffer the library allocates.  The caller passes the max-projection in and
// the candidate array and count out.
//
// The scratch array is a file-scope __device__ array: every GPU that loads
// the library holds it (512 KiB) until the process exits.  Every call shares
// it and it keeps the last call's contents; each call overwrites every entry
// it reads.  Calls that overlap on the GPU (different streams, or different
// host threads on the same device) race on it and must be serialised by the
// caller.  The device address of the array is looked up once per device, on
// that device's first call (with the device current), so that first call
// should be made before any CUDA stream capture starts.  The address is kept
// for the life of the process: after cudaDeviceReset on a device, this entry
// point must not be called on that device again in the same process (the
// kept address would no longer belong to the new context).
#include <mutex>

#include "jerk_internal.h"

namespace jerk {
namespace {

constexpr int kCellsPerBlock = 2048;
constexpr int kThreads = 256;                       // 8 cells per thread
constexpr int64_t kMaxCells = (int64_t)1 << 27;     // largest n_cells accepted
constexpr int kMaxBlocks = (int)(kMaxCells / kCellsPerBlock);   // 65536

// per-block peak counts, then exclusive offsets; entry kMaxBlocks = total
__device__ __align__(256) unsigned long long g_peak_scratch[kMaxBlocks + 1];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long *g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ float mval(unsigned long long x) { return __uint_as_float((unsigned)(x >> 32)); }

// the peak rule of the library: M(p) > theta, M(p) > M(p-1), M(p) >= M(p+1),
// a missing neighbour counting as -inf
__device__ __forceinline__ bool is_peak(const unsigned long long *M, int64_t n, int64_t p, float theta) {
    const float v = mval(M[p]);
    if (!(v > theta)) return false;
    const float l = p > 0 ? mval(M[p - 1]) : -3.402823466e38f;
    const float r = p + 1 < n ? mval(M[p + 1]) : -3.402823466e38f;
    return v > l && v >= r;
}

__device__ __forceinline__ int block_exclusive_scan(int x, int *total) {
    __shared__ int warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int s = lane < kThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    const int before = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[kThreads / 32 - 1];
    __syncthreads();
    return before + incl - x;
}

// 1. peaks per block of cells
__global__ void __launch_bounds__(kThreads) count_kernel(const unsigned long long *M, int64_t n, float theta,
                                                         unsigned long long *scratch) {
    const int64_t base = (int64_t)blockIdx.x * kCellsPerBlock;
    int c = 0;
    for (int i = threadIdx.x; i < kCellsPerBlock; i += kThreads) {
        const int64_t p = base + i;
        if (p < n && is_peak(M, n, p, theta)) ++c;
    }
    int total;
    block_exclusive_scan(c, &total);
    if (threadIdx.x == 0) scratch[blockIdx.x] = (unsigned long long)total;
}

// 2. exclusive prefix sum of the block counts (one CTA), total into d_count
__global__ void __launch_bounds__(1024) scan_kernel(unsigned long long *scratch, int nblk, int64_t *d_count) {
    __shared__ unsigned long long part[1024];
    const int per = (nblk + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(nblk, b0 + per);
    unsigned long long s = 0;
    for (int b = b0; b < b1; ++b) s += scratch[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int i = 0; i < 1024; ++i) {
            const unsigned long long v = part[i];
            part[i] = run;
            run += v;
        }
        scratch[nblk] = run;
        *d_count = (int64_t)run;
    }
    __syncthreads();
    unsigned long long run = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        const unsigned long long v = scratch[b];
        scratch[b] = run;
        run += v;
    }
}

struct GridArgs {
    int32_t stage, zmax, dz, wmax, dw, nz, T;   // T = nz * nw templates
};

// 3. write the records in cell order at the block's offset
__global__ void __launch_bounds__(kThreads) write_kernel(const unsigned long long *M, int64_t n, float theta,
                                                         const unsigned long long *scratch, GridArgs g,
                                                         jerk_candidate *out, int64_t cap) {
    const int64_t base = (int64_t)blockIdx.x * kCellsPerBlock;
    // each thread owns 8 consecutive cells so that the scan keeps cell order
    const int64_t p0 = base + (int64_t)threadIdx.x * (kCellsPerBlock / kThreads);
    unsigned flags = 0;
    int c = 0;
#pragma unroll
    for (int i = 0; i < kCellsPerBlock / kThreads; ++i) {
        const int64_t p = p0 + i;
        if (p < n && is_peak(M, n, p, theta)) {
            flags |= 1u << i;
            ++c;
        }
    }
    int total;
    int pos = block_exclusive_scan(c, &total);
    const int64_t off = (int64_t)scratch[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kCellsPerBlock / kThreads; ++i) {
        if (!((flags >> i) & 1u)) continue;
        const int64_t k = off + pos++;
        if (k >= cap) continue;
        const int64_t p = p0 + i;
        const unsigned long long x = M[p];
        const int t = (int)(0xFFFFFFFFu - (unsigned)(x & 0xFFFFFFFFull));
        jerk_candidate rec;
        rec.p = p;
        rec.r = (double)p / 2.0;
        // a cell that no template reached (or a stale value) decodes to a t
        // outside the grid: reported as the library's candidates do
        const bool on_grid = t >= 0 && t < g.T;
        rec.t = t;
        rec.z_idx = on_grid ? t % g.nz : -1;
        rec.w_idx = on_grid ? t / g.nz : -1;
        rec.stage = g.stage;
        rec.z = on_grid ? (float)(-g.zmax + rec.z_idx * g.dz) : 0.f;
        rec.w = on_grid ? (float)(-g.wmax + rec.w_idx * g.dw) : 0.f;
        rec.power = mval(x);
        rec.item = 0;
        out[k] = rec;
    }
}

}  // namespace
}  // namespace jerk

extern "C" jerk_status jerk_peaks_noalloc(const uint64_t *d_maxproj, int64_t n_cells, float theta, int32_t stage,
                                          int32_t zmax, int32_t dz, int32_t wmax, int32_t dw,
                                          jerk_candidate *d_out, int64_t cap, int64_t *d_count, void *stream) {
    using namespace jerk;
    if (!d_maxproj || !d_count || n_cells < 1 || cap < 0 || (cap > 0 && !d_out)) return JERK_EINVAL;
    if (n_cells > kMaxCells) return JERK_EINVAL;   // beyond the fixed scratch array
    if (dz <= 0 || dw <= 0 || zmax < 0 || wmax < 0 || zmax % dz || wmax % dw || stage < 1) return JERK_EINVAL;
    if ((int64_t)(2 * (int64_t)zmax / dz + 1) * (2 * (int64_t)wmax / dw + 1) > INT32_MAX) return JERK_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return JERK_ECUDA;
    unsigned long long *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_peak_scratch) != cudaSuccess || !ptr) return JERK_ECUDA;
            g_scratch_addr[dev] = (unsigned long long *)ptr;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = (int)((n_cells + kCellsPerBlock - 1) / kCellsPerBlock);
    GridArgs g;
    g.stage = stage;
    g.zmax = zmax;
    g.dz = dz;
    g.wmax = wmax;
    g.dw = dw;
    g.nz = 2 * zmax / dz + 1;
    g.T = g.nz * (2 * wmax / dw + 1);
    const unsigned long long *M = (const unsigned long long *)d_maxproj;
    count_kernel<<<nblk, kThreads, 0, st>>>(M, n_cells, theta, scratch);
    scan_kernel<<<1, 1024, 0, st>>>(scratch, nblk, d_count);
    write_kernel<<<nblk, kThreads, 0, st>>>(M, n_cells, theta, scratch, g, d_out, cap);
    return cudaGetLastError() == cudaSuccess ? JERK_OK : JERK_ECUDA;
}
