// Tile-pass kernel: many gates per pass over the state vector.
//
// Section 2.1 (Figure 3) applies a gate to every pair of states that differ in
// the target bit.  Any set S of b qubits splits the 2^M vector into 2^(M-b)
// independent tiles of 2^b amplitudes (all indices that agree outside S), and
// every gate whose target lies in S maps each tile onto itself.  A pass loads
// one tile into shared memory, applies a whole run of such gates to it in
// circuit order, and writes it back: one read and one write of the vector for
// the run instead of one per gate.
//
// S always holds the L lowest qubits (so a tile is made of contiguous runs of
// 2^L amplitudes, which keeps device-memory access coalesced) and up to
// kMaxTileHigh chosen higher qubits.  Controls outside S are constant over a
// tile (the gate is skipped for tiles where they are not all one); diagonal
// gates may target a qubit outside S, which makes them one factor per tile
// (K_SCALE).  Runs of phase gates are applied at once as a phase polynomial
// (K_PHRUN).  The pass may read from one vector and write to another.
#include "cx.cuh"
#include "qsim_internal.h"
#include "tile_ops.cuh"

namespace qs {
namespace {

template <typename T2>
__device__ void tile_phase_run(T2 *s, int n, const TilePassDesc &d, uint64_t tile,
                               const unsigned char *__restrict__ rec, RunSmem<TurnT<T2>> &rs) {
    using Turn = TurnT<T2>;
    const Turn *Q = phase_run_setup<Turn>(d, tile, rec, rs);
    const int bl = d.b < 7 ? d.b : 7;
    const Turn kt = rs.kt;
    const uint32_t lomask = (1u << bl) - 1;
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
        const Turn phi = kt + rs.lin_lo[u & lomask] + rs.lin_hi[u >> bl] + __ldg(Q + u);
        s[u] = cmul(expi_turns(phi), s[u]);
    }
}

// Insert the op's enumeration bits (ascending positions, given values) into p.
template <typename T2>
__device__ __forceinline__ uint32_t expand_op(uint32_t p, const TileOp<T2> &op) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k < op.npos) {
            const int q = op.pos[k];
            p = ((p >> q) << (q + 1)) | (p & ((1u << q) - 1)) | (uint32_t((op.posval >> k) & 1) << q);
        }
    }
    return p;
}

__device__ __forceinline__ float2 tab_mul(const unsigned char *tab, uint32_t e, float2 x) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(tab) + e);
    return cmulx(make_float2(t.x, t.y), make_float2(t.z, t.w), x);
}
__device__ __forceinline__ double2 tab_mul(const unsigned char *tab, uint32_t e, double2 x) {
    const double2 t = __ldg(reinterpret_cast<const double2 *>(tab) + e);
    return cmul(t, x);
}

template <typename T2>
__device__ __forceinline__ void tile_apply(T2 *s, int n, const TileOp<T2> &op, uint64_t base, uint64_t tile,
                                           const TilePassDesc &d, const unsigned char *runs,
                                           RunSmem<TurnT<T2>> &rs) {
    const uint32_t kind = op.kind;
    if (kind == K_PHRUN) {
        tile_phase_run(s, n, d, tile, runs + op.gsel, rs);
        return;
    }
    const int cnt = n >> op.npos;
    if (kind == K_SCALE || kind == K_PHASE1 || kind == K_DIAG) {
        // diagonal: only the enumerated amplitudes change
        T2 f0 = op.u[0], l0 = op.ul[0], f1 = op.u[3], l1 = op.ul[3];
        if (kind == K_SCALE && (base & op.gsel)) {
            f0 = f1;
            l0 = l1;
        }
        const uint32_t tb = 1u << op.tl;
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint32_t i = expand_op(uint32_t(p), op);
            const bool up = kind == K_PHASE1 || (kind == K_DIAG && (i & tb));
            s[i] = up ? cmulx(f1, l1, s[i]) : cmulx(f0, l0, s[i]);
        }
        return;
    }
    const uint32_t tb = 1u << op.tl;
    if (kind == K_SWAPX) {
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint32_t i = expand_op(uint32_t(p), op);
            const T2 x = s[i];
            s[i] = s[i | tb];
            s[i | tb] = x;
        }
        return;
    }
    const T2 u00 = op.u[0], u01 = op.u[1], u10 = op.u[2], u11 = op.u[3];
    const T2 l00 = op.ul[0], l01 = op.ul[1], l10 = op.ul[2], l11 = op.ul[3];
    if (op.tab_off) {  // the preceding phase gates, applied first
        const unsigned char *tab = runs + op.tab_off;
        const bool one0 = op.tflags & 1;
        const int tw = op.tw;
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            const uint32_t i = expand_op(uint32_t(p), op);
            uint32_t idx = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < tw) idx |= ((i >> op.tpos[k]) & 1u) << k;
            T2 x = s[i], y = s[i | tb];
            if (!one0) x = tab_mul(tab, idx << 1, x);
            y = tab_mul(tab, (idx << 1) | 1u, y);
            s[i] = cmad2x(u00, l00, x, u01, l01, y);
            s[i | tb] = cmad2x(u10, l10, x, u11, l11, y);
        }
        return;
    }
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
        const uint32_t i = expand_op(uint32_t(p), op);
        const T2 x = s[i], y = s[i | tb];
        s[i] = cmad2x(u00, l00, x, u01, l01, y);
        s[i | tb] = cmad2x(u10, l10, x, u11, l11, y);
    }
}

template <typename R>
__global__ void __launch_bounds__(512) k_tile_pass(typename CxT<R>::T *dst, const typename CxT<R>::T *src,
                                                   TilePassDesc d, const TileOp<typename CxT<R>::T> *__restrict__ ops,
                                                   const unsigned char *__restrict__ runs, uint64_t ntiles,
                                                   int ops_in_smem) {
    using T2 = typename CxT<R>::T;
    constexpr int V = CxT<R>::kVec;  // amplitudes per 16-byte access
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *s = reinterpret_cast<T2 *>(smem_raw);
    __shared__ uint64_t hoff[1 << kMaxTileHigh];
    __shared__ RunSmem<TurnT<T2>> rs;

    const int n = 1 << d.b;
    const uint32_t lowmask = (1u << d.L) - 1;
    const TileOp<T2> *op_tab = ops + d.op_begin;
    if (ops_in_smem) {  // stage the pass's ops once per block
        TileOp<T2> *so = reinterpret_cast<TileOp<T2> *>(smem_raw + size_t(n) * sizeof(T2));
        const int4 *g4 = reinterpret_cast<const int4 *>(op_tab);
        int4 *s4 = reinterpret_cast<int4 *>(so);
        const int n4 = int(d.op_count * sizeof(TileOp<T2>) / 16);
        for (int k = threadIdx.x; k < n4; k += blockDim.x) s4[k] = g4[k];
        op_tab = so;
    }
    for (int k = threadIdx.x; k < (1 << d.nh); k += blockDim.x) {
        uint64_t off = 0;
        for (int j = 0; j < d.nh; ++j)
            if ((k >> j) & 1) off |= uint64_t(1) << d.hpos[j];
        hoff[k] = off;
    }
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint64_t base = 0;
        for (int j = 0; j < d.nout; ++j)
            if ((tile >> j) & 1) base |= uint64_t(1) << d.opos[j];
        __syncthreads();  // hoff and ops ready; the previous tile's stores have read s
        for (int u = threadIdx.x * V; u < n; u += blockDim.x * V) {
            const uint64_t g = base | hoff[u >> d.L] | (uint32_t(u) & lowmask);
            if constexpr (V == 2) {
                const float4 v = *reinterpret_cast<const float4 *>(src + g);
                *reinterpret_cast<float4 *>(s + u) = v;
            } else {
                s[u] = src[g];
            }
        }
        __syncthreads();
        for (int k = 0; k < d.op_count; ++k) {
            const TileOp<T2> &op = op_tab[k];
            if ((base & op.gmask) != op.gmask) continue;  // uniform over the block
            tile_apply(s, n, op, base, tile, d, runs, rs);
            __syncthreads();
        }
        for (int u = threadIdx.x * V; u < n; u += blockDim.x * V) {
            const uint64_t g = base | hoff[u >> d.L] | (uint32_t(u) & lowmask);
            if constexpr (V == 2) {
                *reinterpret_cast<float4 *>(dst + g) = *reinterpret_cast<const float4 *>(s + u);
            } else {
                dst[g] = s[u];
            }
        }
    }
}

}  // namespace

int tile_max_bits(qsim_prec prec) { return prec == QSIM_C64 ? 13 : 12; }

int tile_prepare(qsim_prec prec) {
    static int configured[64][2];  // per device
    int dev = 0;
    QS_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && configured[dev][prec]) return QSIM_OK;
    const int maxdyn = 64 * 1024 + kTileOpSmemBytes;
    if (prec == QSIM_C64)
        QS_CUDA(cudaFuncSetAttribute(k_tile_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn));
    else
        QS_CUDA(cudaFuncSetAttribute(k_tile_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn));
    if (dev < 64) configured[dev][prec] = 1;
    return QSIM_OK;
}

int launch_tile_pass(void *dst, const void *src, int M, qsim_prec prec, const TilePassDesc &d,
                     const void *ops_dev, const void *runs_dev, cudaStream_t s) {
    const uint64_t ntiles = uint64_t(1) << (M - d.b);
    const size_t op_bytes = size_t(d.op_count) * (prec == QSIM_C64 ? sizeof(TileOp<float2>) : sizeof(TileOp<double2>));
    const int ops_in_smem = op_bytes <= size_t(kTileOpSmemBytes) ? 1 : 0;
    const size_t smem = (size_t(1) << d.b) * amp_bytes(prec) + (ops_in_smem ? op_bytes : 0);
    // >= 256 threads: the phase-run set-up uses threads 0..255
    const int threads = d.b >= 10 ? 512 : 256;
    if (int rc = tile_prepare(prec)) return rc;
    int per_sm = int((220 * 1024) / (smem + 5120));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2048 / threads) per_sm = 2048 / threads;
    uint64_t grid = uint64_t(num_sms()) * per_sm;
    if (grid > ntiles) grid = ntiles;
    const unsigned char *runs = static_cast<const unsigned char *>(runs_dev);
    if (prec == QSIM_C64) {
        k_tile_pass<float><<<unsigned(grid), threads, smem, s>>>(
            static_cast<float2 *>(dst), static_cast<const float2 *>(src), d,
            static_cast<const TileOp<float2> *>(ops_dev), runs, ntiles, ops_in_smem);
    } else {
        k_tile_pass<double><<<unsigned(grid), threads, smem, s>>>(
            static_cast<double2 *>(dst), static_cast<const double2 *>(src), d,
            static_cast<const TileOp<double2> *>(ops_dev), runs, ntiles, ops_in_smem);
    }
    QS_CHECK_LAUNCH("tile pass launch");
    return QSIM_OK;
}

}  // namespace qs
