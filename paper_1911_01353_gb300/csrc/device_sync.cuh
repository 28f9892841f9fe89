// Device-side synchronisation helpers shared by the filter kernels: shared
// addresses, mbarriers, TMA bulk copies and bounded waits.
#pragma once

#include <stdint.h>

namespace jerk {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one elected thread: expect `bytes` and start the bulk global -> shared copy
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// asynchronous global -> shared copy of 4 or 8 bytes (no register holds the
// value); visible to the issuing thread after cp_async_wait_all, to the other
// threads after a barrier that follows it
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// plain arrival (release): one of the barrier's expected arrivals
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for phase `parity` of `bar`, giving up after limit_ns of %globaltimer
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// the filter kernels' wait: give up after ~1 s
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    return mbar_wait_for(bar, parity, 1000000000ull);
}

// Bounds checks of the debug build (compiled with -DJERK_CHECKS): a failing
// check adds one to chk[0], records its site in chk[1] if it is the first,
// and returns false so that the caller skips the access.  In the release
// build every check is the constant true and costs nothing.
#ifdef JERK_CHECKS
__device__ __forceinline__ bool dev_check(bool ok, long long *chk, int site) {
    if (!ok && chk && atomicAdd(reinterpret_cast<unsigned long long *>(chk), 1ull) == 0ull) chk[1] = site;
    return ok;
}
#define JERK_CHECK(ok, chk, site) ::jerk::dev_check((ok), (chk), (site))
#else
#define JERK_CHECK(ok, chk, site) true
#endif

// OR of `pred` over the `n` threads of named barrier `id` (also a barrier)
__device__ __forceinline__ bool named_any(int id, int n, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

}  // namespace jerk
