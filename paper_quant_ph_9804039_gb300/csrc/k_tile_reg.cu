// Tile passes with register rounds (complex64).
//
// The tile of a pass (Section 2.1's pair rule restricted to 2^b amplitudes,
// see k_tile.cu) is split further: a round picks RB of the tile's qubits (its
// slot qubits) and every one of the block's 256 threads holds, in registers,
// the 2^RB amplitudes of its index that differ only in those qubits.  Every
// gate of the round targets a slot qubit, so its pairs lie inside one
// thread's registers; controls and diagonal gates on any qubit are evaluated
// from each amplitude's index.  A round costs one load and one store of each
// amplitude however many gates it holds; the first round of a pass reads
// device memory and the last writes it, and shared memory carries the tile
// between rounds.  Runs of phase gates on tile qubits are one table lookup
// per amplitude (K_TAB: unit-modulus float entries, one complex multiply),
// longer runs that reach outside the tile a phase polynomial (K_PHRUN).
// Other gate entries are hi + lo floats (compensated complex64, see cx.cuh);
// Hadamards, exact or with a small error, defer their 1/sqrt 2.
#include "cx.cuh"
#include "qsim_internal.h"
#include "tile_ops.cuh"

namespace qs {
namespace {

constexpr int kThreads = 1 << kRegThreadBits;
constexpr int kThreadsPerBlock = kThreads;

template <int RB>
struct Slots {
    static constexpr int S = 1 << RB;
    float2 x[S];
};

// Shared-memory position of tile index i: the low 4 bits are XORed with the
// next 4, so that the 32 lanes of a warp fall on different banks also when a
// round's slot qubits are the tile's lowest.
__device__ __forceinline__ uint32_t swz(uint32_t i) { return i ^ ((i >> 4) & 0xFu); }

// Per-tile state of a phase-polynomial record (K_PHRUN), double-buffered:
// consecutive records of a block alternate between the two copies, so the
// one barrier inside each set-up also orders the writes of a record against
// the reads of the record two before it.
struct PhRunState {
    uint32_t cl[2][16];  // linear coefficient of each tile-local bit, given the tile's outside bits
    uint32_t ktw[2][8];  // the tile's constant, one partial sum per warp
};

// Phi(i) = c0 + sum_q c_q i_q + sum_{q<r} w_qr i_q i_r (turns of 2^-32) on
// the tile with outside bits `tile`: tile-local bit t gets
// cl[t] = c_{q_t} + sum over set outside bits k of w[q_t][r_k] (warp t mod 8,
// one outside bit per lane, summed with a warp reduction), and the constant
// sums c_{r_k} + w[r_k][r_k2] over set outside bits k <= k2 (all threads, one
// (k, k2) pair each).  All threads of the block call it.
__device__ __forceinline__ void phrun_setup(const TilePassDesc &d, uint64_t tile, const unsigned char *__restrict__ rec,
                                            PhRunState &ps, int buf) {
    const PhaseRunHdr h = *reinterpret_cast<const PhaseRunHdr *>(rec);
    const int M = int(h.M);
    const uint32_t *c = reinterpret_cast<const uint32_t *>(rec + sizeof(PhaseRunHdr)) + 1;
    const uint32_t *w = c + M;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nout = d.nout;
    const bool set = lane < nout && ((tile >> lane) & 1);
    const int r = lane < nout ? d.opos[lane] : 0;
    for (int t = warp; t < d.b; t += kThreadsPerBlock / 32) {
        const int q = t < d.L ? t : d.hpos[t - d.L];
        const uint32_t v = __reduce_add_sync(0xffffffffu, set ? __ldg(w + q * M + r) : 0u);
        if (lane == 0) ps.cl[buf][t] = v + __ldg(c + q);
    }
    uint32_t kv = 0;
    for (int p = threadIdx.x; p < nout * nout; p += kThreadsPerBlock) {
        const int k = p / nout, k2 = p - k * nout;
        if (k2 < k || !((tile >> k) & 1) || !((tile >> k2) & 1)) continue;
        kv += k2 == k ? __ldg(c + d.opos[k]) : __ldg(w + d.opos[k] * M + d.opos[k2]);
    }
    kv = __reduce_add_sync(0xffffffffu, kv);
    if (lane == 0) ps.ktw[buf][warp] = kv;
    __syncthreads();
}

// Pair update on slot bit K: pairs (c, c | 2^K) of this thread's slots, for
// the lower slots c in op.smask (controls on slot qubits are folded into the
// mask, controls on other tile qubits into op.nmask, tested by the caller).
template <int RB, int K, bool SWAP, bool REAL, bool ALL>
__device__ __forceinline__ void pairs(Slots<RB> &v, const RegOp &op) {
    constexpr int S = 1 << RB;
    const uint32_t sm = op.smask;
#pragma unroll
    for (int c = 0; c < S; ++c) {
        if (c & (1 << K)) continue;
        if (!ALL && !((sm >> c) & 1u)) continue;
        const int c1 = c | (1 << K);
        const float2 a = v.x[c], b = v.x[c1];
        if (SWAP) {
            v.x[c] = b;
            v.x[c1] = a;
        } else if (REAL) {  // real entries: (u + ul) a + (w + wl) b per component
            v.x[c] = make_float2(fmaf(op.u[0].x, a.x, fmaf(op.u[1].x, b.x, fmaf(op.ul[0].x, a.x, op.ul[1].x * b.x))),
                                 fmaf(op.u[0].x, a.y, fmaf(op.u[1].x, b.y, fmaf(op.ul[0].x, a.y, op.ul[1].x * b.y))));
            v.x[c1] = make_float2(fmaf(op.u[2].x, a.x, fmaf(op.u[3].x, b.x, fmaf(op.ul[2].x, a.x, op.ul[3].x * b.x))),
                                  fmaf(op.u[2].x, a.y, fmaf(op.u[3].x, b.y, fmaf(op.ul[2].x, a.y, op.ul[3].x * b.y))));
        } else {
            v.x[c] = cmad2x(op.u[0], op.ul[0], a, op.u[1], op.ul[1], b);
            v.x[c1] = cmad2x(op.u[2], op.ul[2], a, op.u[3], op.ul[3], b);
        }
    }
}

// A Hadamard with an error, without its factor 1/sqrt 2: (a, b) <- (a + b +
// e0 a + e1 b, a - b + e2 a + e3 b) on slot bit K.
template <int RB, int K>
__device__ __forceinline__ void pairs_nhad(Slots<RB> &v, const RegOp &op) {
    const float e0 = op.u[0].x, e1 = op.u[1].x, e2 = op.u[2].x, e3 = op.u[3].x;
#pragma unroll
    for (int c = 0; c < (1 << RB); ++c) {
        if (c & (1 << K)) continue;
        const int c1 = c | (1 << K);
        const float2 a = v.x[c], b = v.x[c1];
        v.x[c] = make_float2(fmaf(e0, a.x, fmaf(e1, b.x, a.x + b.x)), fmaf(e0, a.y, fmaf(e1, b.y, a.y + b.y)));
        v.x[c1] = make_float2(fmaf(e2, a.x, fmaf(e3, b.x, a.x - b.x)), fmaf(e2, a.y, fmaf(e3, b.y, a.y - b.y)));
    }
}

// Hadamard without its factor: (a, b) <- (a + b, a - b) on slot bit K.
template <int RB, int K>
__device__ __forceinline__ void pairs_had(Slots<RB> &v) {
#pragma unroll
    for (int c = 0; c < (1 << RB); ++c) {
        if (c & (1 << K)) continue;
        const int c1 = c | (1 << K);
        const float2 a = v.x[c], b = v.x[c1];
        v.x[c] = make_float2(a.x + b.x, a.y + b.y);
        v.x[c1] = make_float2(a.x - b.x, a.y - b.y);
    }
}

template <int RB>
__device__ __forceinline__ void apply_op(Slots<RB> &v, const RegOp &op, uint32_t i0, const RoundDesc &R,
                                         uint64_t base, uint64_t tile, const TilePassDesc &d,
                                         const unsigned char *__restrict__ runs, PhRunState &ps, int &nrun) {
    constexpr int S = 1 << RB;
    if (op.code == RC_PHRUN) {  // every thread reaches the synchronisation inside
        // Phi(i0 | slots c) = Phi(i0) + sum_{k in c} (cl[pos_k] + Q(i0 | bit_k) - Q(i0)) + Q(slots c):
        // five exponentials per thread, the slot-only factors e^{i Q(slots c)} precomputed.
        const unsigned char *rec = runs + op.gsel;
        const int buf = nrun++ & 1;
        phrun_setup(d, tile, rec, ps, buf);
        const PhaseRunHdr h = *reinterpret_cast<const PhaseRunHdr *>(rec);
        const uint32_t *Q = reinterpret_cast<const uint32_t *>(rec + h.q_offset);
        const uint32_t q0 = __ldg(Q + i0);
        uint32_t phi = __ldg(reinterpret_cast<const uint32_t *>(rec + sizeof(PhaseRunHdr))) + q0;
#pragma unroll
        for (int j = 0; j < kThreadsPerBlock / 32; ++j) phi += ps.ktw[buf][j];
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if ((i0 >> t) & 1) phi += ps.cl[buf][t];
        float2 e[S];
        e[0] = expi_turns(phi);
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            const uint32_t pk = R.pos[k];
            const float2 dk = expi_turns(ps.cl[buf][pk] + __ldg(Q + (i0 | (1u << pk))) - q0);
#pragma unroll
            for (int c = 0; c < (1 << k); ++c) e[c | (1 << k)] = cmul(e[c], dk);
        }
        const float2 *f = reinterpret_cast<const float2 *>(runs + op.tab_off);
#pragma unroll
        for (int c = 0; c < S; ++c) v.x[c] = cmul(cmul(e[c], __ldg(f + c)), v.x[c]);
        return;
    }
    if ((i0 & op.nmask) != op.nmask) return;  // a control (or the target) outside the slots is 0
    const uint32_t code = op.code;
    const uint32_t sm = op.smask;
    // an if-tree of small switches, the common kinds first (the Hadamard is
    // taken by the caller): one switch over every code was measured at about
    // twice the cost per op
    if (code == RC_TAB) {
        uint32_t g = 0;  // index bits held by the thread's base index
        for (int j = 0; j < op.tw; ++j) g |= ((i0 >> op.tpos[j]) & 1u) << j;
        const float4 *tab = reinterpret_cast<const float4 *>(runs + op.tab_off);
#pragma unroll
        for (int c = 0; c < S; ++c) {
            if (!((sm >> c) & 1u)) continue;
            const float4 t = __ldg(tab + (g | op.cidx[c]));  // unit-modulus float entry (the lo part unused)
            v.x[c] = cmul(make_float2(t.x, t.y), v.x[c]);
        }
        return;
    }
#define QS_PAIR_SWITCH(BASE, SWAP, REAL)                                                     \
    switch (code - BASE) {                                                                    \
        case 0: pairs<RB, 0, SWAP, REAL, true>(v, op); break;                                 \
        case 1: pairs<RB, 1, SWAP, REAL, true>(v, op); break;                                 \
        case 2: pairs<RB, 2, SWAP, REAL, true>(v, op); break;                                 \
        case 3: if constexpr (RB > 3) pairs<RB, 3, SWAP, REAL, true>(v, op); break;           \
        case 4: pairs<RB, 0, SWAP, REAL, false>(v, op); break;                                \
        case 5: pairs<RB, 1, SWAP, REAL, false>(v, op); break;                                \
        case 6: pairs<RB, 2, SWAP, REAL, false>(v, op); break;                                \
        default: if constexpr (RB > 3) pairs<RB, 3, SWAP, REAL, false>(v, op); break;         \
    }
    if (code < RC_RDENSE) {
        QS_PAIR_SWITCH(RC_DENSE, false, false)
        return;
    }
    if (code < RC_SWAP) {
        QS_PAIR_SWITCH(RC_RDENSE, false, true)
        return;
    }
    if (code < RC_PHASE_ALL) {
        QS_PAIR_SWITCH(RC_SWAP, true, false)
        return;
    }
#undef QS_PAIR_SWITCH
    if (code == RC_PHASE_ALL) {
#pragma unroll
        for (int c = 0; c < S; ++c) v.x[c] = cmulx(op.u[3], op.ul[3], v.x[c]);
    } else if (code == RC_PHASE) {
#pragma unroll
        for (int c = 0; c < S; ++c)
            if ((sm >> c) & 1u) v.x[c] = cmulx(op.u[3], op.ul[3], v.x[c]);
    } else if (code == RC_DIAG) {
        const bool up_thread = (i0 & op.tbn) != 0;
#pragma unroll
        for (int c = 0; c < S; ++c) {
            if (!((sm >> c) & 1u)) continue;
            const bool up = op.tbn ? up_thread : ((op.tsel >> c) & 1u);
            v.x[c] = up ? cmulx(op.u[3], op.ul[3], v.x[c]) : cmulx(op.u[0], op.ul[0], v.x[c]);
        }
    } else if (code == RC_SCALE) {
        const bool up = (base & op.gsel) != 0;
        const float2 f = up ? op.u[3] : op.u[0], fl = up ? op.ul[3] : op.ul[0];
#pragma unroll
        for (int c = 0; c < S; ++c)
            if ((sm >> c) & 1u) v.x[c] = cmulx(f, fl, v.x[c]);
    }
}

template <int RB>
__global__ void __launch_bounds__(kThreads, 3) k_tile_reg(float2 *dst, const float2 *src, TilePassDesc d,
                                                          const RegOp *__restrict__ ops,
                                                          const RoundDesc *__restrict__ rounds,
                                                          const unsigned char *__restrict__ runs, uint64_t ntiles) {
    constexpr int S = 1 << RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *s = reinterpret_cast<float2 *>(smem_raw);
    RegOp *sops = reinterpret_cast<RegOp *>(smem_raw + (d.round_count > 1 ? (size_t(1) << d.b) * sizeof(float2) : 0));
    __shared__ uint64_t hoff[1 << kMaxTileHigh];
    __shared__ PhRunState ps;
    int nrun = 0;  // K_PHRUN records met so far (uniform over the block)
    const int tid = threadIdx.x;
    {  // the pass's ops, staged once
        const int4 *g4 = reinterpret_cast<const int4 *>(ops + d.op_begin);
        int4 *s4 = reinterpret_cast<int4 *>(sops);
        const int n4 = int(d.op_count * sizeof(RegOp) / 16);
        for (int k = tid; k < n4; k += kThreads) s4[k] = g4[k];
    }
    for (int k = tid; k < (1 << d.nh); k += kThreads) {
        uint64_t off = 0;
        for (int j = 0; j < d.nh; ++j)
            if ((k >> j) & 1) off |= uint64_t(1) << d.hpos[j];
        hoff[k] = off;
    }
    __syncthreads();
    const uint32_t lowmask = (1u << d.L) - 1;
    Slots<RB> v;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint64_t base = 0;
        for (int j = 0; j < d.nout; ++j)
            if ((tile >> j) & 1) base |= uint64_t(1) << d.opos[j];
        for (int rd = 0; rd < d.round_count; ++rd) {
            const RoundDesc R = rounds[d.round_begin + rd];
            uint32_t i0 = uint32_t(tid);
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                const int q = R.pos[k];
                i0 = ((i0 >> q) << (q + 1)) | (i0 & ((1u << q) - 1));
            }
            uint32_t dep[S];
#pragma unroll
            for (int c = 0; c < S; ++c) {
                uint32_t o = 0;
#pragma unroll
                for (int k = 0; k < RB; ++k)
                    if (c & (1 << k)) o |= 1u << R.pos[k];
                dep[c] = o;
            }
            if (rd == 0) {
#pragma unroll
                for (int c = 0; c < S; ++c) {
                    const uint32_t i = i0 | dep[c];
                    v.x[c] = src[base | hoff[i >> d.L] | (i & lowmask)];
                }
            } else {
#pragma unroll
                for (int c = 0; c < S; ++c) v.x[c] = s[swz(i0 | dep[c])];
            }
            for (int k = R.op_begin; k < R.op_begin + R.op_count; ++k) {
                const RegOp &op = sops[k];
                const uint32_t code = op.code;
                if (code >= RC_HAD) {  // the commonest op, before any other test (no controls by construction)
                    switch (code - RC_HAD) {
                        case 0: pairs_had<RB, 0>(v); break;
                        case 1: pairs_had<RB, 1>(v); break;
                        case 2: pairs_had<RB, 2>(v); break;
                        case 3: if constexpr (RB > 3) pairs_had<RB, 3>(v); break;
                        case 4: pairs_nhad<RB, 0>(v, op); break;
                        case 5: pairs_nhad<RB, 1>(v, op); break;
                        case 6: pairs_nhad<RB, 2>(v, op); break;
                        default: if constexpr (RB > 3) pairs_nhad<RB, 3>(v, op); break;
                    }
                    continue;
                }
                if (op.gmask && (base & op.gmask) != op.gmask) continue;  // uniform over the block
                apply_op<RB>(v, op, i0, R, base, tile, d, runs, ps, nrun);
            }
            if (rd + 1 == d.round_count) {
                if (d.pscale_on) {  // the pass's deferred Hadamard factors, compensated
#pragma unroll
                    for (int c = 0; c < S; ++c)
                        v.x[c] = make_float2(fmaf(v.x[c].x, d.pscale_hi, v.x[c].x * d.pscale_lo),
                                             fmaf(v.x[c].y, d.pscale_hi, v.x[c].y * d.pscale_lo));
                }
#pragma unroll
                for (int c = 0; c < S; ++c) {
                    const uint32_t i = i0 | dep[c];
                    dst[base | hoff[i >> d.L] | (i & lowmask)] = v.x[c];
                }
            } else {
                __syncthreads();  // every thread has read its amplitudes of the previous round
#pragma unroll
                for (int c = 0; c < S; ++c) s[swz(i0 | dep[c])] = v.x[c];
                __syncthreads();
            }
        }
    }
}

}  // namespace

int tile_reg_prepare() {
    static int configured[64];
    int dev = 0;
    QS_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && configured[dev]) return QSIM_OK;
    QS_CUDA(cudaFuncSetAttribute(k_tile_reg<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024 + kTileOpSmemBytes));
    QS_CUDA(cudaFuncSetAttribute(k_tile_reg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024 + kTileOpSmemBytes));
    if (dev < 64) configured[dev] = 1;
    return QSIM_OK;
}

int launch_tile_reg(void *dst, const void *src, int M, const TilePassDesc &d, const void *ops_dev,
                    const void *rounds_dev, const void *runs_dev, cudaStream_t s) {
    const int RB = d.b - kRegThreadBits;
    if (RB < 3 || RB > 4) {
        set_error("register rounds need a tile of %d..%d qubits", kRegThreadBits + 3, kRegThreadBits + 4);
        return QSIM_EINVAL;
    }
    if (int rc = tile_reg_prepare()) return rc;
    const uint64_t ntiles = uint64_t(1) << (M - d.b);
    const size_t smem = (d.round_count > 1 ? (size_t(1) << d.b) * sizeof(float2) : 0) + size_t(d.op_count) * sizeof(RegOp);
    int per_sm = 0;
    if (RB == 3) QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_reg<3>, kThreads, smem));
    else QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_reg<4>, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    uint64_t grid = uint64_t(num_sms()) * per_sm;  // one wave of resident blocks, each looping over tiles
    if (grid > ntiles) grid = ntiles;
    const RegOp *ops = static_cast<const RegOp *>(ops_dev);
    const RoundDesc *rounds = static_cast<const RoundDesc *>(rounds_dev);
    const unsigned char *runs = static_cast<const unsigned char *>(runs_dev);
    if (RB == 3)
        k_tile_reg<3><<<unsigned(grid), kThreads, smem, s>>>(static_cast<float2 *>(dst), static_cast<const float2 *>(src),
                                                             d, ops, rounds, runs, ntiles);
    else
        k_tile_reg<4><<<unsigned(grid), kThreads, smem, s>>>(static_cast<float2 *>(dst), static_cast<const float2 *>(src),
                                                             d, ops, rounds, runs, ntiles);
    QS_CHECK_LAUNCH("register tile pass launch");
    return QSIM_OK;
}

}  // namespace qs
