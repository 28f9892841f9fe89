// Tensor memory as per-thread storage for the FP32 filter's constant factors.
//
// Each SM has 256 KB of tensor memory (128 lanes x 512 columns of 32 bits),
// read by tcgen05.ld on its own path, not through the shared-memory pipe.
// Warp w of a CTA reaches lanes 32 (w % 4) .. 32 (w % 4) + 31, one lane per
// thread, so a thread can keep private words there: warps w, w + 4, w + 8,
// w + 12 share a lane range and take disjoint column ranges.  The FP32 filter
// keeps the twiddle factors of its inverse transform there (the same for
// every template), which takes their reads off the shared-memory pipe that
// bounds it.
#pragma once

#include <stdint.h>

namespace jerk {

// one warp: allocate `ncols` columns (a power of two >= 32) and write their
// base address to the shared-memory word `slot`; then give up the right to
// allocate more, so that other CTAs on the SM are not held up
__device__ __forceinline__ void tmem_alloc_warp(uint32_t slot_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// the warp that allocated: free the columns (every thread's tensor-memory
// accesses ordered before it by a barrier between tmem_fence_before and
// tmem_fence_after)
__device__ __forceinline__ void tmem_dealloc_warp(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive columns of this thread's lane from x (warp-collective)
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&x)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(x[0])), "r"(__float_as_uint(x[1])), "r"(__float_as_uint(x[2])),
                 "r"(__float_as_uint(x[3])), "r"(__float_as_uint(x[4])), "r"(__float_as_uint(x[5])),
                 "r"(__float_as_uint(x[6])), "r"(__float_as_uint(x[7]))
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Start loading 8 consecutive columns of this thread's lane into r
// (warp-collective).  The registers are not valid until tmem_wait_ld8(r),
// which also waits for every earlier load of this thread.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

// wait for this thread's loads; the operands tie r to the wait, so that no
// use of r is scheduled before it
__device__ __forceinline__ void tmem_wait_ld8(uint32_t (&r)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
}

}  // namespace jerk
