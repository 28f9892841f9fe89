// Harmonic-row stores shared by the FP32 and the tensor-core filters.
//
// The harmonic sum (Sec. 3) reads, for every fundamental cell p and harmonic
// h, the power of template t_h at cell q = h p.  The filters write those
// powers as decimated rows ("slots"): row entry (h, off, len) of a template
// holds its power at cells q = h p, p < len, at a.slots + off + p.  A filter
// first stages one segment's power row in shared memory (swizzled by swzf),
// then every thread of the segment stores its share of each entry coalesced.
#pragma once

#include "device_sync.cuh"
#include "jerk_internal.h"

namespace jerk {

// float swizzle for the staged power row: bits 5-7 of the cell flipped into
// bits 1-3.  The FP32 filter's digit-reversed writes (lanes differ in cell
// bits 0 and 4-7) then meet 32 distinct banks, the h = 2 reads at most 3.  A
// group of 4 cells stays in one 16-byte block, its two pairs swapped when
// bit 5 of the cell is set (row4 undoes it).
__device__ __forceinline__ int swzf(int a) { return a ^ (((a >> 5) & 7) << 1); }

// cells 4g .. 4g + 3 of the staged row, in order, from one 16-byte load
__device__ __forceinline__ float4 row4(const float *pw, int g) {
    const int a = 4 * g;
    const float4 v = *reinterpret_cast<const float4 *>(pw + (swzf(a) & ~3));
    return ((a >> 5) & 1) ? make_float4(v.z, v.w, v.x, v.y) : v;
}

// Store the staged power row `pw` of one template (cell c of the segment at
// pw[swzf(c)], the segment starting at cell s0) into its n row entries, with
// the segment's `nt` threads (this one is j).  sb[h - 1] holds the first and
// last p whose cell h p lies in the segment and in the spectrum.  `site` names
// the store in the bounds-checked build.
__device__ __forceinline__ void store_rows(const ConvArgs &a, const RowEntries &en, int n, const float *pw,
                                           const int (*sb)[2], int s0, int j, int nt, int site) {
    for (int e = 0; e < n; ++e) {
        const int h = en.h[e];
        const int64_t off = en.off[e];
        float *dst = a.slots + off;
        const int len = (int)en.len[e];
        const int pf = sb[h - 1][0];
        const int pl = min(sb[h - 1][1], len - 1);
        if (pl < pf) continue;                                // this segment is past the row's end
        if (h == 1) {
            // p = s0 + v: whole groups of 4 (s0 and the segment's valid length
            // are multiples of 4 and the row is 128-byte aligned), then the
            // ragged end one by one
            const int n4 = (pl - pf + 1) >> 2;
            for (int g = j; g < n4; g += nt)
                if (JERK_CHECK(off + pf + 4 * g + 3 < a.slot_cap, a.chk, site))
                    *reinterpret_cast<float4 *>(dst + pf + 4 * g) = row4(pw, g);
            for (int p = pf + 4 * n4 + j; p <= pl; p += nt)
                if (JERK_CHECK(off + p < a.slot_cap, a.chk, site)) dst[p] = pw[swzf(p - s0)];
        } else {
            for (int p = pf + j; p <= pl; p += nt)
                if (JERK_CHECK(off + p < a.slot_cap, a.chk, site)) dst[p] = pw[swzf(h * p - s0)];
        }
    }
}

}  // namespace jerk
