// One gate applied to a tile of 2^b amplitudes held in shared memory
// (Section 2.1, Figure 3, restricted to the tile): shared by the tile-pass
// kernel and the error-trajectory kernel.
#pragma once

#include "cx.cuh"
#include "qsim_internal.h"

namespace qs {

// Insert the bits of `mask` (set to one) into x, lowest first.
__device__ __forceinline__ uint32_t insert_ones(uint32_t x, uint32_t mask) {
    while (mask) {
        const int pos = __ffs(mask) - 1;
        mask &= mask - 1;
        const uint32_t lo = x & ((1u << pos) - 1);
        x = ((x >> pos) << (pos + 1)) | lo | (1u << pos);
    }
    return x;
}

// kind: K_DENSE, K_DIAG, K_PHASE1, K_SWAPX (target tl inside the tile) or
// K_SCALE (diagonal gate whose target is outside the tile; `up` = that
// target's bit in this tile).  lmask = control bits inside the tile.  u / ul
// = matrix entries U00, U01, U10, U11 (hi and lo parts for complex64).
// Called by all threads of the block; the caller synchronises afterwards.
template <typename T2>
__device__ __forceinline__ void tile_gate(T2 *s, int n, uint32_t kind, uint32_t tl, uint32_t lmask, bool up,
                                          const T2 *u, const T2 *ul) {
    if (kind == K_SCALE) {
        const T2 f = up ? u[3] : u[0], fl = up ? ul[3] : ul[0];
        const int cnt = n >> __popc(lmask);
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint32_t i = insert_ones(uint32_t(p), lmask);
            s[i] = cmulx(f, fl, s[i]);
        }
        return;
    }
    const uint32_t tb = 1u << tl;
    if (kind == K_PHASE1) {  // only states with the target and local controls set change
        const uint32_t m = lmask | tb;
        const int cnt = n >> __popc(m);
        const T2 u11 = u[3], l11 = ul[3];
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint32_t i = insert_ones(uint32_t(p), m);
            s[i] = cmulx(u11, l11, s[i]);
        }
        return;
    }
    if (kind == K_DIAG) {
        const T2 u00 = u[0], u11 = u[3], l00 = ul[0], l11 = ul[3];
        const int cnt = n >> __popc(lmask);
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint32_t i = insert_ones(uint32_t(p), lmask);
            s[i] = (i & tb) ? cmulx(u11, l11, s[i]) : cmulx(u00, l00, s[i]);
        }
        return;
    }
    const int half = n >> 1;
    if (kind == K_SWAPX) {
        for (int p = threadIdx.x; p < half; p += blockDim.x) {
            const uint32_t i = uint32_t(insert0(uint64_t(p), int(tl)));
            if ((i & lmask) != lmask) continue;
            const T2 x = s[i];
            s[i] = s[i | tb];
            s[i | tb] = x;
        }
        return;
    }
    const T2 u00 = u[0], u01 = u[1], u10 = u[2], u11 = u[3];
    const T2 l00 = ul[0], l01 = ul[1], l10 = ul[2], l11 = ul[3];
    for (int p = threadIdx.x; p < half; p += blockDim.x) {
        const uint32_t i = uint32_t(insert0(uint64_t(p), int(tl)));
        if ((i & lmask) != lmask) continue;
        const T2 x = s[i], y = s[i | tb];
        s[i] = cmad2x(u00, l00, x, u01, l01, y);
        s[i | tb] = cmad2x(u10, l10, x, u11, l11, y);
    }
}

}  // namespace qs
