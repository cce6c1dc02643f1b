// Fused dense blocks on the tensor cores (tcgen05, kind::f16, FP32 accumulate).
//
// Section 2.1 applies a 2x2 block to every pair of states that differ in one
// bit.  A run of gates acting on k qubits B = {b_0 < ... < b_{k-1}} multiplies
// to one dense 2^k x 2^k unitary U (built on the host in FP64), which acts on
// every sub-vector of 2^k amplitudes that differ only in those k bits.  With
// x the sub-vector in interleaved real form (re, im of each amplitude),
// y = R x where R is the 2^(k+1) square real form of U
// (R[2a][2b] = Re U[a][b], R[2a][2b+1] = -Im U[a][b], R[2a+1][2b] = Im U[a][b],
// R[2a+1][2b+1] = Re U[a][b]).  For 128 sub-vectors at a time this is the
// matrix product D (128 x 2^(k+1)) = X (128 x 2^(k+1)) R^T: the one dense
// contraction of the simulator, run on the tensor cores.
//
// Precision: complex64 amplitudes, FP32 accumulation.  Both operands are
// split into FP16 pairs, v = hi + lo (11 + 11 significant bits), and
// D = X_lo R_hi + X_hi R_lo + X_hi R_hi (the lo*lo term is below 2^-22
// relative).  FP16 has a narrow exponent range, so every sub-vector is scaled
// by a power of two that puts its largest component just below 2^15 before
// the split (and R by 2^8); the epilogue multiplies the scale back out, which
// is exact.  The tensor core's FP32 accumulation truncates, which shrinks
// every output by a fraction of an ulp on average; over many blocks that bias
// would show in the norm and the fidelity.  A unitary block preserves the norm
// of every sub-vector, so for blocks the planner has checked to be unitary the
// epilogue rescales each output sub-vector to its input norm (the correction
// applied as v + v c with c = (|x|^2 - |y|^2) / (2 |y|^2)), which removes the
// bias and leaves unbiased rounding.
//
// Tile: the k block qubits plus F = the 12 - k lowest other qubits, 4096
// amplitudes numbered by a tile-local index u whose bits are the qubits of
// B u F in ascending order.  B u F always holds qubits 0..6, so a tile is a
// set of contiguous runs of >= 128 amplitudes, loaded by bulk TMA copies
// (cp.async.bulk).  Sub-vector m (0 .. 2^(12-k) - 1) and block combination a
// sit at u = posA[a] | posM[m]; the 2^(12-k) sub-vectors form 2^(5-k) MMA
// row blocks of 128.  A tile is loaded in 16-byte asynchronous copies
// (cp.async) by all lanes of the producer warp: bulk copies of the 1 KiB runs
// of a tile on high qubits were measured at half the bandwidth.
//
// Per CTA (persistent over tiles, one per SM, 384 threads), warp-specialised
// and pipelined over tiles:
//   warps 0..2   producers: asynchronous copies of a tile into one of 3 or 4
//                input stages, each lane arriving on the stage's mbarrier
//                when its copies have landed (a lane's 16-byte pieces and
//                their offsets from the tile's base are fixed per CTA and
//                computed once: per tile the producers were issue-bound);
//   warp 3       MMA: 12 tcgen05.mma per tile (3 products x row blocks x
//                K steps of 16) into one of 2 TMEM accumulators (64 columns
//                each), committed to mbarriers;
//   warps 4..7   split: each thread owns one sub-vector row per row block,
//                reads its 2^k amplitudes (in a lane-skewed order, so the
//                warp's reads and writes fall on distinct banks), scales,
//                splits and writes X_hi, X_lo into one of 2 operand stages in
//                the canonical K-major swizzled layout the MMA reads;
//   warps 8..11  epilogue: each thread reads its row of the accumulator
//                (tcgen05.ld), removes the scale, renormalises and stores
//                the amplitudes: straight to device memory when a warp's
//                stores fill whole 32-byte sectors (the block avoids qubits 0
//                and 1; then a fourth input stage takes the staging tile's
//                shared memory), otherwise into an XOR-swizzled staging tile
//                of which each warp copies out its own quarter in 16-byte
//                pieces (no barrier between the four warps).
// The split warps release an input stage as soon as the tile is in their
// registers, before converting it.
// Every mbarrier wait is bounded: the main loops' waits by wait_ns (2 s by
// default, qsim_opts.wait_us), the drain waits at the end always by 2 s of
// globaltimer.  On a timeout the CTA records QSIM_ETIMEOUT in the status
// word, the other roles leave their loops, the producer waits for its copies
// in flight (cp.async.wait_all, and the R image's bulk copy), the MMA warp for
// both commits of its last tile, and the CTA frees its TMEM and returns.
#include <cuda_fp16.h>

#include "cx.cuh"
#include "qsim_internal.h"

namespace qs {
namespace {

constexpr int kProd = 3;                    // producer warps (one per scheduler, 0..2)
constexpr int kMmaWarp = kProd;             // the MMA warp
constexpr int kSplit0 = kProd + 1;          // first of the 4 split warps
constexpr int kEpi0 = kProd + 5;            // first of the 4 epilogue warps
constexpr int kThreads = 32 * (kProd + 9);  // 12 warps
constexpr int kMaxIn = 4;      // input stages (3 with a staging tile for the output, 4 without)
constexpr int kNA = 2;         // operand stages = accumulator stages
constexpr int kTileAmps = 1 << kFusedTileBits;
constexpr uint32_t kInBytes = kTileAmps * 8;
constexpr uint32_t kABytes = kTileAmps * 4;  // one of X_hi / X_lo for the whole tile (FP16 pairs)
constexpr uint32_t kAccCols = 64;            // TMEM columns of one accumulator stage
constexpr uint32_t kTmemCols = kNA * kAccCols;
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
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
// Bounded wait on an mbarrier phase of the main loops; false once limit_ns
// have passed or the CTA is aborting.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, const volatile int *abort, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (globaltimer() - t0 > limit_ns) return false;
    }
    return true;
}
// The same wait by every lane of a warp, with one outcome for all of them
// (the warp stays converged for the .sync.aligned tcgen05 instructions).
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, const volatile int *abort,
                                          uint64_t limit_ns) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort, limit_ns)) != 0;
}
// Drain wait at the end of a CTA (copies or MMAs still in flight): always the
// full kWaitNs, whatever the main loops' limit, and not cut short by abort.
__device__ __forceinline__ void drain_wait(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > kWaitNs) break;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// arrive on bar once this thread's earlier cp.async copies have landed
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor, K-major, swizzled rows of W bytes
// (W = 128, 64 or 32: layout 2, 4 or 6), 8-row groups 8 W bytes apart,
// descriptor version 1.
template <int W>
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
    constexpr uint64_t layout = W == 128 ? 2 : (W == 64 ? 4 : 6);
    return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(1) << 16) | (uint64_t((8 * W) >> 4) << 32) |
           (uint64_t(1) << 46) | (layout << 61);
}
// Instruction descriptor of kind::f16: D f32, A and B f16, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x N consecutive 32-bit columns of TMEM (thread = lane), issued
// without waiting; tmem_wait_ld completes every load issued before it.
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float *v);
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float *v) {
    uint32_t *r = reinterpret_cast<uint32_t *>(v);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, float *v) {
    tmem_ld<16>(taddr, v);
    tmem_ld<16>(taddr + 16, v + 16);
}
template <>
__device__ __forceinline__ void tmem_ld<64>(uint32_t taddr, float *v) {
    tmem_ld<32>(taddr, v);
    tmem_ld<32>(taddr + 32, v + 32);
}
// Completes every TMEM load issued before it; the empty statements after it
// tie the loaded registers to this point, so no use moves above the wait.
template <int N>
__device__ __forceinline__ void tmem_wait_ld(float *v) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < N; i += 8)
        asm volatile("" : "+f"(v[i]), "+f"(v[i + 1]), "+f"(v[i + 2]), "+f"(v[i + 3]), "+f"(v[i + 4]), "+f"(v[i + 5]),
                     "+f"(v[i + 6]), "+f"(v[i + 7]));
}

template <int KF, bool DIRECT>
struct Cfg {
    static constexpr int NIN = DIRECT ? 4 : 3;         // input stages
    static constexpr int NA = 1 << KF;                 // amplitudes per sub-vector
    static constexpr int KR = 2 * NA;                  // reals per sub-vector (MMA K and N)
    static constexpr int W = KR * 2;                   // bytes of one operand row (FP16)
    static constexpr int NRB = 1 << (5 - KF);          // row blocks of 128 sub-vectors per tile
    static constexpr int NROWS = 128 * NRB;            // sub-vectors per tile
    static constexpr uint32_t RB_BYTES = 128 * W;      // one row block of one operand
    static constexpr uint32_t B_BYTES = KR * KR * 2;   // one of R_hi / R_lo
    static constexpr int KSTEPS = KR / 16;             // MMA K = 16 (32 bytes)
    // dynamic shared memory: inputs, operands (hi, lo per stage), R, staging
    static constexpr uint32_t OFF_IN = 0;
    static constexpr uint32_t OFF_A = OFF_IN + NIN * kInBytes;
    static constexpr uint32_t OFF_B = OFF_A + kNA * 2 * kABytes;
    static constexpr uint32_t OFF_OUT = OFF_B + 2 * (B_BYTES < 1024 ? 1024 : B_BYTES);
    static constexpr uint32_t SMEM = 1024 + OFF_OUT + (DIRECT ? 0 : kInBytes);
};

struct SmemCtl {
    uint64_t full_in[kMaxIn], empty_in[kMaxIn];
    uint64_t full_a[kNA], empty_a[kNA];
    uint64_t full_acc[kNA], empty_acc[kNA];
    uint64_t bar_r;
    uint64_t runoff[32];                  // device offset of run r of a tile (tile 0)
    uint64_t runoff2[32];                 // device offset of tile-local index 128 j (tile 0)
    uint64_t qdev[4][16];                 // staged copy-out: device offset of piece it of quarter q (lane 0)
    uint32_t qidx[4][16];                 // staged copy-out: tile index of piece it of quarter q (lane 0)
    uint64_t gA[32];                      // device offset of combination a (sub-vector 0, tile 0)
    uint32_t tmem;
    int abort;
    uint32_t swA8[32];                    // 8 * swz(posA[a]): staging byte offset of combination a
    uint16_t posM[1 << kFusedRowBits];    // u of sub-vector m
    float2 rowinfo[kNA][1 << kFusedRowBits];  // per sub-vector: (|x|^2, 1 / total scale)
};

// XOR swizzle of the staging tile (8-byte amplitudes): bits [0,4) ^= bits [r, r+4).
__device__ __forceinline__ uint32_t stg_swz(uint32_t u, int r) { return u ^ ((u >> r) & 15u); }

template <int KF, bool DIRECT>
__global__ void __launch_bounds__(kThreads, 1)
    k_fused_tc(float2 *dst, const float2 *src, FusedDesc d, const __half *__restrict__ rimg, uint64_t ntiles,
               int *status, uint64_t wait_ns) {
    using C = Cfg<KF, DIRECT>;
    constexpr int kNIn = C::NIN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // 1024-byte aligned, derived from the shared array by pointer arithmetic so
    // that every access through it stays a shared-memory access (no aliasing
    // with device memory for the compiler to assume)
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ SmemCtl ctl;
    volatile int *abort = &ctl.abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nrun = 1 << d.nrb;
    const uint32_t run_amps = 1u << d.runbits;
    for (int m = tid; m < C::NROWS; m += kThreads) ctl.posM[m] = d.posM[m];
    if (tid < C::NA) ctl.swA8[tid] = 8u * stg_swz(d.posA[tid], d.outsh);
    if (tid < 32) ctl.runoff2[tid] = d.runoff2[tid];
    if (!DIRECT && tid < 64) {  // the staged copy-out's offsets, the same for every tile
        const uint32_t b5 = d.posM[32], b6 = d.posM[64];
        const int q = tid >> 4, it = tid & 15;
        uint32_t u = uint32_t(it * 64);
        u = ((u & ~(b5 - 1u)) << 1) | (u & (b5 - 1u));
        u = ((u & ~(b6 - 1u)) << 1) | (u & (b6 - 1u));
        u |= ((q & 1) ? b5 : 0u) | ((q & 2) ? b6 : 0u);
        ctl.qidx[q][it] = u;
        ctl.qdev[q][it] = d.runoff2[u >> 7] + (u & 127u);
    }
    if (tid < C::NA) {  // tile-local index posA[a] -> device offset
        const uint32_t u = d.posA[tid];
        uint64_t off = u & (run_amps - 1);
        for (int b = 0; b < d.nrb; ++b)
            if (((u >> d.runbits) >> b) & 1) off |= uint64_t(1) << d.rpos[b];
        ctl.gA[tid] = off;
    }
    if (tid < nrun) {
        uint64_t off = 0;
        for (int b = 0; b < d.nrb; ++b)
            if ((tid >> b) & 1) off |= uint64_t(1) << d.rpos[b];
        ctl.runoff[tid] = off;
    }
    if (tid == 0) {
        for (int b = 0; b < kNIn; ++b) {
            mbar_init(&ctl.full_in[b], 32 * kProd);
            mbar_init(&ctl.empty_in[b], 4);
        }
        for (int b = 0; b < kNA; ++b) {
            mbar_init(&ctl.full_a[b], 4);
            mbar_init(&ctl.empty_a[b], 1);
            mbar_init(&ctl.full_acc[b], 1);
            mbar_init(&ctl.empty_acc[b], 4);
        }
        mbar_init(&ctl.bar_r, 1);
        ctl.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc(&ctl.tmem, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl.tmem;
    const uint64_t n_local = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    // device offset of the CTA's i-th tile: lane j contributes outside bit j (a
    // warp OR-reduction, every lane of the warp calls it)
    const int my_opos = lane < d.nout ? d.opos[lane] : 0;
    auto tile_base = [&](uint64_t i) {
        const uint64_t tile = blockIdx.x + i * gridDim.x;
        const uint64_t mine = (lane < d.nout && ((tile >> lane) & 1)) ? uint64_t(1) << my_opos : 0;
        const uint32_t lo = __reduce_or_sync(0xffffffffu, uint32_t(mine));
        const uint32_t hi = __reduce_or_sync(0xffffffffu, uint32_t(mine >> 32));
        return (uint64_t(hi) << 32) | lo;
    };
    bool ok = true;

    if (warp < kProd) {
        // ------------------------------------------------------------ producer
        // the producer warps (one per scheduler) copy the tile in 16-byte
        // pieces (cp.async), each lane arriving on the stage's barrier once its
        // copies have landed
        uint64_t issued = 0;
        const int ptid = warp * 32 + lane;
        if (warp == 0 && lane == 0) {
            unsigned char *Bs = sm + C::OFF_B;
            const uint32_t bstride = C::B_BYTES < 1024 ? 1024 : C::B_BYTES;
            mbar_expect_tx(&ctl.bar_r, 2 * C::B_BYTES);
            bulk_g2s(Bs, rimg, C::B_BYTES, &ctl.bar_r);
            bulk_g2s(Bs + bstride, rimg + C::B_BYTES / 2, C::B_BYTES, &ctl.bar_r);
        }
        const uint32_t rmask = run_amps - 1;
        // this lane's 16-byte pieces of a tile (piece c = ptid + 96 j holds
        // tile amplitudes 2c, 2c + 1): their byte offsets from the tile's base,
        // the same for every tile, so they are computed once
        constexpr int kPieces = (kTileAmps / 2 + 32 * kProd - 1) / (32 * kProd);
        uint64_t poff[kPieces];
#pragma unroll
        for (int j = 0; j < kPieces; ++j) {
            const int c = ptid + j * 32 * kProd;
            const uint32_t u = 2u * uint32_t(c < kTileAmps / 2 ? c : 0);
            poff[j] = 8u * (ctl.runoff[u >> d.runbits] + (u & rmask));
        }
        for (uint64_t i = 0; i < n_local; ++i) {
            const int s = int(i % kNIn);
            if (i >= kNIn && !warp_wait(&ctl.empty_in[s], uint32_t(((i / kNIn) & 1) ^ 1), abort, wait_ns)) {
                ok = false;
                break;
            }
            const uint64_t base = tile_base(i);
            unsigned char *buf = sm + C::OFF_IN + size_t(s) * kInBytes;
            const unsigned char *srcb = reinterpret_cast<const unsigned char *>(src + base);
#pragma unroll
            for (int j = 0; j < kPieces; ++j) {
                const int c = ptid + j * 32 * kProd;
                if (j + 1 < kPieces || c < kTileAmps / 2) cp_async16(buf + 16u * uint32_t(c), srcb + poff[j]);
            }
            cp_async_arrive(&ctl.full_in[s]);
            issued = i + 1;
        }
        cp_async_wait_all();
        if (!ok) {
            if (lane == 0) atomicExch(status, QSIM_ETIMEOUT);
            ctl.abort = 1;
        }
        if (warp == 0 && lane == 0) drain_wait(&ctl.bar_r, 0);  // the R image's bulk copy has landed
        (void)issued;
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ----------------------------------------------------------------- MMA
        uint64_t done = 0;  // tiles whose MMAs were issued
        if (lane == 0) {
            ok = mbar_wait(&ctl.bar_r, 0, abort, wait_ns);
            const uint32_t bh = smem_u32(sm + C::OFF_B);
            const uint32_t bl = bh + (C::B_BYTES < 1024 ? 1024 : C::B_BYTES);
            constexpr uint32_t IDESC = idesc_f16(128, C::KR);
            for (uint64_t i = 0; ok && i < n_local; ++i) {
                const int t = int(i % kNA);
                const uint32_t ph = uint32_t((i / kNA) & 1);
                if (!mbar_wait(&ctl.full_a[t], ph, abort, wait_ns)) { ok = false; break; }
                if (i >= kNA && !mbar_wait(&ctl.empty_acc[t], ph ^ 1, abort, wait_ns)) { ok = false; break; }
                tc_fence_after();
                const uint32_t ah = smem_u32(sm + C::OFF_A + uint32_t(t) * 2 * kABytes);
                const uint32_t al = ah + kABytes;
                const uint32_t As[3] = {al, ah, ah}, Bs[3] = {bh, bl, bh};  // small products first
#pragma unroll
                for (int rb = 0; rb < C::NRB; ++rb) {
                    const uint32_t dcol = tmem + uint32_t(t) * kAccCols + uint32_t(rb * C::KR);
#pragma unroll
                    for (int pr = 0; pr < 3; ++pr) {
#pragma unroll
                        for (int ks = 0; ks < C::KSTEPS; ++ks) {
                            const uint64_t ad = sw_desc<C::W>(As[pr] + uint32_t(rb) * C::RB_BYTES + uint32_t(ks) * 32);
                            const uint64_t bd = sw_desc<C::W>(Bs[pr] + uint32_t(ks) * 32);
                            mma_f16(dcol, ad, bd, IDESC, (pr | ks) != 0);
                        }
                    }
                }
                mma_commit(&ctl.empty_a[t]);
                mma_commit(&ctl.full_acc[t]);
                done = i + 1;
            }
            if (!ok) {
                atomicExch(status, QSIM_ETIMEOUT);
                ctl.abort = 1;
            }
            if (done > 0) {  // the last MMAs and both their commits must be complete before TMEM is freed
                const uint64_t j = done - 1;
                drain_wait(&ctl.empty_a[j % kNA], uint32_t((j / kNA) & 1));
                drain_wait(&ctl.full_acc[j % kNA], uint32_t((j / kNA) & 1));
            }
        }
        __syncwarp();
    } else if (warp < kEpi0) {
        // --------------------------------------------------------------- split
        const int sw = warp - kSplit0;
        const uint32_t g = d.skew[lane];
        const uint32_t pAg = d.posA[g];
        uint32_t posA8[C::NA];
#pragma unroll
        for (int a = 0; a < C::NA; ++a) posA8[a] = 8u * d.posA[a];
        for (uint64_t i = 0; i < n_local; ++i) {
            const int s_in = int(i % kNIn), t = int(i % kNA);
            const uint32_t ph = uint32_t((i / kNA) & 1);
            ok = warp_wait(&ctl.full_in[s_in], uint32_t((i / kNIn) & 1), abort, wait_ns);
            if (ok && i >= kNA) ok = warp_wait(&ctl.empty_a[t], ph ^ 1, abort, wait_ns);
            if (ok && i >= kNA) ok = warp_wait(&ctl.empty_acc[t], ph ^ 1, abort, wait_ns);
            if (!ok) break;
            const unsigned char *in = sm + C::OFF_IN + size_t(s_in) * kInBytes;
            unsigned char *ahi = sm + C::OFF_A + uint32_t(t) * 2 * kABytes;
#pragma unroll 1
            for (int rb = 0; rb < C::NRB; ++rb) {
                const int rho = 32 * sw + lane;
                const int m = rb * 128 + rho;
                const uint32_t lin = 8u * (pAg ^ ctl.posM[m]);
                float2 x[C::NA];
                float mx = 0.f;
#pragma unroll
                for (int s = 0; s < C::NA; ++s) {
                    x[s] = *reinterpret_cast<const float2 *>(in + (posA8[s] ^ lin));
                    mx = fmaxf(mx, fmaxf(fabsf(x[s].x), fabsf(x[s].y)));
                }
                if (rb + 1 == C::NRB) {  // the tile is in registers: its input stage can be refilled
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ctl.empty_in[s_in]);
                }
                // scale 2^es puts the largest component in [2^14, 2^15); rows below
                // 2^-104 keep es = 118, so that 2^-es-8 stays a normal float
                const int e = int((__float_as_uint(mx) >> 23) & 255u) - 127;
                int es = 14 - e;
                if (es > 118) es = 118;
                const float scale = __uint_as_float(uint32_t(es + 127) << 23);
                const float inv = __uint_as_float(uint32_t(127 - es - 8) << 23);  // 2^-es * 2^-8 (R's scale)
                float sx = 0.f;  // |x|^2 in scaled units (no overflow or underflow)
                // operand row rho of row block rb: amplitude a at bytes 4a, 16-byte chunks swizzled
                uint32_t swr;
                if constexpr (C::W == 128) swr = uint32_t(rho & 7);
                else if constexpr (C::W == 64) swr = uint32_t((rho >> 1) & 3);
                else swr = uint32_t((rho >> 2) & 1);
                const uint32_t cl = (uint32_t(rho) * C::W) ^ (swr << 4) ^ (4u * g);
                unsigned char *rowb = ahi + uint32_t(rb) * C::RB_BYTES;
                if constexpr (DIRECT) {
#pragma unroll
                    for (int s = 0; s < C::NA; ++s) {
                        const float2 xs = make_float2(x[s].x * scale, x[s].y * scale);
                        sx = fmaf(xs.x, xs.x, fmaf(xs.y, xs.y, sx));
                        const __half2 h = __float22half2_rn(xs);
                        const float2 hf = __half22float2(h);
                        const __half2 l = __float22half2_rn(make_float2(xs.x - hf.x, xs.y - hf.y));
                        const uint32_t off = cl ^ (4u * uint32_t(s));
                        *reinterpret_cast<__half2 *>(rowb + off) = h;
                        *reinterpret_cast<__half2 *>(rowb + kABytes + off) = l;
                    }
                } else {
                    // staged blocks (bound by the epilogue warps, which share
                    // their schedulers with these): packed float pairs, one
                    // instruction for the real and imaginary parts, |x|^2 as two
                    // partial sums added at the end (measured 5.7 -> 6.05 TB/s
                    // per staged block; the direct blocks ran 3 % slower so)
                    float2 sx2 = make_float2(0.f, 0.f);
                    const float2 scale2 = make_float2(scale, scale), mone2 = make_float2(-1.f, -1.f);
#pragma unroll
                    for (int s = 0; s < C::NA; ++s) {
                        const float2 xs = __fmul2_rn(x[s], scale2);
                        sx2 = __ffma2_rn(xs, xs, sx2);
                        const __half2 h = __float22half2_rn(xs);
                        const float2 hf = __half22float2(h);
                        const __half2 l = __float22half2_rn(__ffma2_rn(hf, mone2, xs));  // xs - hf, one rounding
                        const uint32_t off = cl ^ (4u * uint32_t(s));
                        *reinterpret_cast<__half2 *>(rowb + off) = h;
                        *reinterpret_cast<__half2 *>(rowb + kABytes + off) = l;
                    }
                    sx = sx2.x + sx2.y;
                }
                ctl.rowinfo[t][m] = make_float2(sx, inv);
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl.full_a[t]);
        }
        if (!ok) {
            if (lane == 0) atomicExch(status, QSIM_ETIMEOUT);
            ctl.abort = 1;
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int qd = warp & 3;  // TMEM lane quadrant of this warp
        const unsigned char *outb = sm + C::OFF_OUT;
        uint64_t rowoff[C::NRB];  // device offset of this thread's rows (direct stores), the same in every tile
#pragma unroll
        for (int rb = 0; rb < C::NRB; ++rb) {
            const uint32_t u = ctl.posM[rb * 128 + 32 * qd + lane];
            rowoff[rb] = ctl.runoff[u >> d.runbits] | (u & (run_amps - 1));
        }
        for (uint64_t i = 0; i < n_local; ++i) {
            const int t = int(i % kNA);
            ok = warp_wait(&ctl.full_acc[t], uint32_t((i / kNA) & 1), abort, wait_ns);
            // the split's row data of this tile (complete, as the MMAs that read its operands are)
            if (ok) ok = warp_wait(&ctl.full_a[t], uint32_t((i / kNA) & 1), abort, wait_ns);
            if (!ok) break;
            tc_fence_after();
            const int rho = 32 * qd + lane;
            float y[C::NRB][C::KR];
            float2 ri[C::NRB];
#pragma unroll
            for (int rb = 0; rb < C::NRB; ++rb) {
                ri[rb] = ctl.rowinfo[t][rb * 128 + rho];
                tmem_ld<C::KR>(tmem + (uint32_t(32 * qd) << 16) + uint32_t(t) * kAccCols + uint32_t(rb * C::KR), y[rb]);
            }
            tmem_wait_ld<C::NRB * C::KR>(&y[0][0]);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl.empty_acc[t]);
#pragma unroll
            for (int rb = 0; rb < C::NRB; ++rb) {
                float sy = 0.f;  // in the split's scaled units: the accumulator carries R's 2^8 too
                if constexpr (DIRECT) {
#pragma unroll
                    for (int j = 0; j < C::KR; ++j) {
                        const float ys = y[rb][j] * (1.0f / 256.0f);
                        sy = fmaf(ys, ys, sy);
                        y[rb][j] *= ri[rb].y;
                    }
                } else {  // packed float pairs, as in the split of staged blocks
                    float2 sy2 = make_float2(0.f, 0.f);
                    const float2 q2 = make_float2(1.0f / 256.0f, 1.0f / 256.0f), inv2 = make_float2(ri[rb].y, ri[rb].y);
#pragma unroll
                    for (int j = 0; j < C::KR; j += 2) {
                        const float2 yv = make_float2(y[rb][j], y[rb][j + 1]);
                        const float2 ys = __fmul2_rn(yv, q2);
                        sy2 = __ffma2_rn(ys, ys, sy2);
                        const float2 yo = __fmul2_rn(yv, inv2);
                        y[rb][j] = yo.x;
                        y[rb][j + 1] = yo.y;
                    }
                    sy = sy2.x + sy2.y;
                }
                if (d.unitary) {
                    const float sx = ri[rb].x;
                    // sqrt(sx/sy) - 1 to first order, kept as a small number: the
                    // bias is a fraction of an ulp, so a scale factor near 1 would
                    // round to exactly 1; v + v c rounds to nearest, unbiased.
                    const float c = (sx > 0.f && sy > 0.f) ? (sx - sy) / (2.f * sy) : 0.f;
                    if constexpr (DIRECT) {
#pragma unroll
                        for (int j = 0; j < C::KR; ++j) y[rb][j] = fmaf(y[rb][j], c, y[rb][j]);
                    } else {
                        const float2 c2 = make_float2(c, c);
#pragma unroll
                        for (int j = 0; j < C::KR; j += 2) {
                            const float2 yv = make_float2(y[rb][j], y[rb][j + 1]);
                            const float2 yo = __ffma2_rn(yv, c2, yv);
                            y[rb][j] = yo.x;
                            y[rb][j + 1] = yo.y;
                        }
                    }
                }
            }
            const uint64_t base = tile_base(i);
            if constexpr (DIRECT) {
                // the 32 rows of a warp are 32 consecutive amplitudes: every store
                // of a combination a writes 256 contiguous bytes, no staging
#pragma unroll
                for (int rb = 0; rb < C::NRB; ++rb) {
                    float2 *drow = dst + base + rowoff[rb];
#pragma unroll
                    for (int a = 0; a < C::NA; ++a) drow[ctl.gA[a]] = make_float2(y[rb][2 * a], y[rb][2 * a + 1]);
                }
            } else {
                // staged: warp qd's rows fill the quarter of the staging tile whose
                // tile bits b5, b6 (those of sub-vector bits 5 and 6) equal qd, and
                // the warp copies that quarter out itself, so the four warps never
                // wait for one another.  b5 and b6 are tile bits 6 and up (the block
                // holds qubit 0 or 1, below them), so a quarter is made of 16 pieces
                // of 64 amplitudes: 16 bytes a lane, each warp store 512 contiguous
                // bytes; the pieces' tile indices and device offsets are tabled once
                // per CTA (computing them per tile cost a fifth of the staged
                // blocks' speed).  The swizzle only mixes bits 0..3 with bits
                // outsh..outsh+3, so it keeps every quarter and every aligned pair.
#pragma unroll
                for (int rb = 0; rb < C::NRB; ++rb) {
                    const uint32_t swm = 8u * stg_swz(ctl.posM[rb * 128 + rho], d.outsh);
#pragma unroll
                    for (int a = 0; a < C::NA; ++a)
                        *reinterpret_cast<float2 *>(const_cast<unsigned char *>(outb) + (ctl.swA8[a] ^ swm)) =
                            make_float2(y[rb][2 * a], y[rb][2 * a + 1]);
                }
                __syncwarp();
                {
                    float2 *dq = dst + base + 2 * lane;
#pragma unroll
                    for (int it0 = 0; it0 < 16; it0 += 8) {  // 8 loads in flight, then their stores
                        float4 v[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const uint32_t u = ctl.qidx[qd][it0 + j] | uint32_t(2 * lane);
                            const uint32_t su = stg_swz(u, d.outsh);
                            float4 w = *reinterpret_cast<const float4 *>(outb + 8u * (su & ~1u));
                            if (su & 1u) w = make_float4(w.z, w.w, w.x, w.y);  // the pair stored swapped
                            v[j] = w;
                        }
#pragma unroll
                        for (int j = 0; j < 8; ++j) *reinterpret_cast<float4 *>(dq + ctl.qdev[qd][it0 + j]) = v[j];
                    }
                }
                __syncwarp();  // the quarter is read before the next tile's rows overwrite it
            }
        }
        if (!ok) {
            if (lane == 0) atomicExch(status, QSIM_ETIMEOUT);
            ctl.abort = 1;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

int fused_prepare() {
    static int configured[64];
    int dev = 0;
    QS_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && configured[dev]) return QSIM_OK;
#define QS_FUSED_ATTR(K, D) \
    QS_CUDA(cudaFuncSetAttribute(k_fused_tc<K, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg<K, D>::SMEM)))
    QS_FUSED_ATTR(3, false);
    QS_FUSED_ATTR(4, false);
    QS_FUSED_ATTR(5, false);
    QS_FUSED_ATTR(3, true);
    QS_FUSED_ATTR(4, true);
    QS_FUSED_ATTR(5, true);
#undef QS_FUSED_ATTR
    if (dev < 64) configured[dev] = 1;
    return QSIM_OK;
}

size_t fused_rimg_halves(int k) { return 2 * size_t(4) << (2 * k); }  // 2 x (2^(k+1))^2

int launch_fused(void *dst, const void *src, int M, const FusedDesc &d, const void *rimg_dev, int *status,
                 cudaStream_t s, uint64_t wait_ns) {
    if (wait_ns == 0) wait_ns = kWaitNs;
    if (int rc = fused_prepare()) return rc;
    const uint64_t ntiles = uint64_t(1) << (M - kFusedTileBits);
    uint64_t grid = uint64_t(num_sms());
    if (grid > ntiles) grid = ntiles;
    float2 *o = static_cast<float2 *>(dst);
    const float2 *i = static_cast<const float2 *>(src);
    const __half *r = static_cast<const __half *>(rimg_dev);
#define QS_FUSED_LAUNCH(K, D) \
    k_fused_tc<K, D><<<unsigned(grid), kThreads, Cfg<K, D>::SMEM, s>>>(o, i, d, r, ntiles, status, wait_ns)
    switch (d.k * 2 + (d.direct ? 1 : 0)) {
        case 6: QS_FUSED_LAUNCH(3, false); break;
        case 7: QS_FUSED_LAUNCH(3, true); break;
        case 8: QS_FUSED_LAUNCH(4, false); break;
        case 9: QS_FUSED_LAUNCH(4, true); break;
        case 10: QS_FUSED_LAUNCH(5, false); break;
        case 11: QS_FUSED_LAUNCH(5, true); break;
        default: set_error("fused block width %d outside [3, 5]", d.k); return QSIM_EINVAL;
    }
#undef QS_FUSED_LAUNCH
    QS_CHECK_LAUNCH("fused tensor-core launch");
    return QSIM_OK;
}

}  // namespace qs
