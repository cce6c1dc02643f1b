// One gate applied to a tile of 2^b amplitudes held in shared memory
// (Section 2.1, Figure 3, restricted to the tile): shared by the tile-pass
// kernel and the error-trajectory kernel.
#pragma once

#include "cx.cuh"
#include "qsim_internal.h"

namespace qs {

template <typename Turn>
struct RunSmem {
    Turn cl[16];       // per-tile linear coefficient of each tile-local bit
    Turn lin_lo[128];  // linear part over local bits [0, 7)
    Turn lin_hi[128];  // linear part over local bits [7, b)
    Turn kt;           // constant of the tile
};

// e^{2 pi i phi / 2^32}: the top 24 bits go through sincospif (exact argument),
// the low 8 bits (< 3.7e-7 rad) as a first-order rotation.
__device__ __forceinline__ float2 expi_turns(uint32_t phi) {
    const int32_t sp = int32_t(phi);
    const float x = float(sp >> 8) * (1.0f / 8388608.0f);  // (phi >> 8) / 2^23, in [-1, 1)
    float sn, cs;
    sincospif(x, &sn, &cs);
    const float r = float(phi & 255u) * 1.4629180792671596e-09f;  // 2 pi / 2^32
    return make_float2(fmaf(-sn, r, cs), fmaf(cs, r, sn));
}
// e^{2 pi i phi / 2^64}
__device__ __forceinline__ double2 expi_turns(uint64_t phi) {
    const double x = double(int64_t(phi)) * (1.0 / 9223372036854775808.0);
    double sn, cs;
    sincospi(x, &sn, &cs);
    return make_double2(cs, sn);
}

// Per-tile set-up of a phase-polynomial record (all threads of the block
// call it; it synchronises): the linear coefficient of every tile-local bit
// given the tile's outside bits, the two linear lookup tables and the tile's
// constant.  Returns the record's quadratic table Q (indexed by the tile-local
// index).  Phi(u) = kt + lin_lo[u & 127] + lin_hi[u >> 7] + Q[u].
template <typename Turn>
__device__ const Turn *phase_run_setup(const TilePassDesc &d, uint64_t tile, const unsigned char *__restrict__ rec,
                                       RunSmem<Turn> &rs) {
    const PhaseRunHdr h = *reinterpret_cast<const PhaseRunHdr *>(rec);
    const int M = int(h.M);
    const Turn *c0p = reinterpret_cast<const Turn *>(rec + sizeof(PhaseRunHdr));
    const Turn *c = c0p + 1;
    const Turn *w = c + M;
    const int b = d.b;
    const int t = threadIdx.x;
    __syncthreads();  // rs may still be read by a previous run
    if (t < b) {  // warp 0: linear coefficient of each tile-local bit, given the tile's outside bits
        const int q = t < d.L ? t : d.hpos[t - d.L];
        Turn v = c[q];
        for (int k = 0; k < d.nout; ++k)
            if ((tile >> k) & 1) v += w[q * M + d.opos[k]];
        rs.cl[t] = v;
    } else if (t >= 32 && t < 64) {  // warp 1: the tile's constant, one outside bit per lane
        Turn v = 0;
        for (int k = t - 32; k < d.nout; k += 32) {
            if (!((tile >> k) & 1)) continue;
            const int r = d.opos[k];
            v += c[r];
            for (int k2 = k + 1; k2 < d.nout; ++k2)
                if ((tile >> k2) & 1) v += w[r * M + d.opos[k2]];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (t == 32) rs.kt = v + *c0p;
    }
    __syncthreads();
    const int bl = b < 7 ? b : 7;
    const int bh = b - bl;
    if (t < (1 << bl)) {
        Turn v = 0;
        for (int j = 0; j < bl; ++j)
            if ((t >> j) & 1) v += rs.cl[j];
        rs.lin_lo[t] = v;
    }
    if (t >= 128 && t - 128 < (1 << bh)) {
        const int v0 = t - 128;
        Turn v = 0;
        for (int j = 0; j < bh; ++j)
            if ((v0 >> j) & 1) v += rs.cl[bl + j];
        rs.lin_hi[v0] = v;
    }
    __syncthreads();
    return reinterpret_cast<const Turn *>(rec + h.q_offset);
}

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
