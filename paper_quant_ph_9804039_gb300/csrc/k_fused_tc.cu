// Fused dense blocks on the tensor cores (tcgen05, kind::tf32).
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
// Precision: complex64 amplitudes, FP32 accumulation.  TF32 keeps 11
// significant bits, so both operands are split, v = hi + lo with hi and lo
// rounded to TF32 (to nearest), and D = X_lo R_hi + X_hi R_lo + X_hi R_hi
// (the lo*lo term is below 2^-22 relative).  The tensor core's FP32
// accumulation truncates, which shrinks every output by a fraction of an ulp
// on average; over many blocks that bias would show in the norm and the
// fidelity.  A unitary block preserves the norm of every sub-vector, so for
// blocks the planner has checked to be unitary the epilogue rescales each
// output sub-vector to its input norm (sums in FP32, rounded to nearest; the
// correction applied as v + v c with c = (|x|^2 - |y|^2) / (2 |y|^2)), which
// removes the bias and leaves unbiased rounding.
//
// Tile: the k block qubits plus F = the 7 lowest other qubits, 2^(k+7)
// amplitudes, numbered by a tile-local index u whose bits are the qubits of
// B u F in ascending order.  B u F always holds qubits 0..6, so a tile is a
// set of contiguous runs of >= 128 amplitudes, moved by bulk TMA copies
// (cp.async.bulk) into and out of shared memory.  Sub-vector m (0..127) and
// block combination a (0..2^k-1) sit at u = posA[a] | posM[m].
//
// Per CTA (persistent over tiles, 256 threads):
//   load   one thread issues the bulk copies of a tile two tiles ahead
//          (three tile buffers), completion on an mbarrier;
//   split  all threads turn the tile into X_hi and X_lo in the canonical
//          K-major 128-byte-swizzled layout that the MMA descriptors read;
//   mma    one thread issues 3 x 2^(k+1)/8 tcgen05.mma (M=128, N=2^(k+1),
//          K=8) into a TMEM accumulator and commits to an mbarrier;
//   store  8 warps read the accumulator (tcgen05.ld, each warp its 32 TMEM
//          lanes and half the columns), write the tile buffer back in tile
//          order, and one thread issues the bulk stores.
// Every mbarrier wait is bounded (2 s of globaltimer); on a timeout the CTA
// records QSIM_ETIMEOUT in the status word, waits (bounded) for its copies in
// flight, frees its TMEM and returns.
#include "cx.cuh"
#include "qsim_internal.h"

namespace qs {
namespace {

constexpr int kMT = 128;       // sub-vectors per tile (MMA M)
constexpr int kThreads = 256;  // 8 warps
constexpr int kNBuf = 3;       // tile buffers
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
// Bounded wait on an mbarrier phase; false once kWaitNs have passed.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > kWaitNs) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
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

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the swizzle atom), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
           (uint64_t(1) << 46) | (uint64_t(2) << 61);
}
// Instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns of TMEM: thread = lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int KF>
struct Cfg {
    static constexpr int NA = 1 << KF;                // amplitudes per sub-vector
    static constexpr int KR = 2 * NA;                 // reals per sub-vector (MMA K and N)
    static constexpr int TILE = NA * kMT;             // amplitudes per tile
    static constexpr uint32_t A_BYTES = kMT * KR * 4;  // one X operand (hi or lo)
    static constexpr uint32_t A_CHUNK = kMT * 128;     // one 128-byte K chunk of X
    static constexpr uint32_t B_BYTES = KR * KR * 4;   // one R operand
    static constexpr uint32_t B_CHUNK = KR * 128;
    static constexpr uint32_t IN_BYTES = TILE * 8;
    static constexpr uint32_t TMEM_COLS = KR < 32 ? 32 : KR;
    static constexpr uint32_t SMEM = 1024 + 2 * A_BYTES + 2 * B_BYTES + kNBuf * IN_BYTES;
};

struct SmemCtl {
    uint64_t bar_load[kNBuf];
    uint64_t bar_mma;
    uint64_t bar_r;
    uint64_t runoff[32];
    uint32_t tmem;
    int abort;
    uint16_t posA[32];
    uint16_t posM[kMT];
    uint8_t decA[2][64];  // a = decA[0][u & 63] | decA[1][u >> 6]
    uint8_t decM[2][64];  // m = decM[0][u & 63] | decM[1][u >> 6]
    float2 red[2][kMT];   // per row and column half: (|x|^2, |y|^2)
};

template <int KF>
__global__ void __launch_bounds__(kThreads, 1)
    k_fused_tc(float2 *dst, const float2 *src, FusedDesc d, const float *__restrict__ rimg, uint64_t ntiles,
               int *status) {
    using C = Cfg<KF>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float *Ahi = reinterpret_cast<float *>(sm);
    float *Alo = reinterpret_cast<float *>(sm + C::A_BYTES);
    float *Bhi = reinterpret_cast<float *>(sm + 2 * C::A_BYTES);
    float *Blo = reinterpret_cast<float *>(sm + 2 * C::A_BYTES + C::B_BYTES);
    float2 *IN = reinterpret_cast<float2 *>(sm + 2 * C::A_BYTES + 2 * C::B_BYTES);
    __shared__ SmemCtl ctl;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nrun = 1 << d.nrb;
    const uint32_t run_amps = 1u << d.runbits;
    if (tid < C::NA) ctl.posA[tid] = d.posA[tid];
    if (tid < kMT) ctl.posM[tid] = d.posM[tid];
    if (tid < 64) {
        ctl.decA[0][tid] = d.decA[0][tid];
        ctl.decA[1][tid] = d.decA[1][tid];
        ctl.decM[0][tid] = d.decM[0][tid];
        ctl.decM[1][tid] = d.decM[1][tid];
    }
    if (tid < nrun) {
        uint64_t off = 0;
        for (int i = 0; i < d.nrb; ++i)
            if ((tid >> i) & 1) off |= uint64_t(1) << d.rpos[i];
        ctl.runoff[tid] = off;
    }
    if (tid == 0) {
        for (int b = 0; b < kNBuf; ++b) mbar_init(&ctl.bar_load[b], 1);
        mbar_init(&ctl.bar_mma, 1);
        mbar_init(&ctl.bar_r, 1);
        ctl.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&ctl.tmem, C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl.tmem;

    const uint64_t n_local = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    auto tile_base = [&](uint64_t i) {
        const uint64_t tile = blockIdx.x + i * gridDim.x;
        uint64_t base = 0;
        for (int j = 0; j < d.nout; ++j)
            if ((tile >> j) & 1) base |= uint64_t(1) << d.opos[j];
        return base;
    };
    auto issue_load = [&](uint64_t i) {  // thread 0 only
        const int b = int(i % kNBuf);
        const uint64_t base = tile_base(i);
        float2 *buf = IN + size_t(b) * C::TILE;
        mbar_expect_tx(&ctl.bar_load[b], C::IN_BYTES);
        for (int r = 0; r < nrun; ++r)
            bulk_g2s(buf + size_t(r) * run_amps, src + base + ctl.runoff[r], run_amps * 8, &ctl.bar_load[b]);
    };

    uint64_t issued = 0;  // tiles whose load was issued
    if (tid == 0) {
        mbar_expect_tx(&ctl.bar_r, 2 * C::B_BYTES);
        bulk_g2s(Bhi, rimg, C::B_BYTES, &ctl.bar_r);
        bulk_g2s(Blo, rimg + C::B_BYTES / 4, C::B_BYTES, &ctl.bar_r);
        for (; issued < n_local && issued < kNBuf - 1; ++issued) issue_load(issued);
    }
    bool ok = mbar_wait(&ctl.bar_r, 0);
    constexpr uint32_t IDESC = idesc_tf32(kMT, C::KR);

    for (uint64_t i = 0; ok && i < n_local; ++i) {
        const int b = int(i % kNBuf);
        float2 *buf = IN + size_t(b) * C::TILE;
        ok = mbar_wait(&ctl.bar_load[b], uint32_t((i / kNBuf) & 1));
        if (__syncthreads_or(!ok)) { ok = false; break; }

        // split: tile order -> X_hi, X_lo (row m, column 2a + re/im), swizzled
        for (int u = tid * 2; u < C::TILE; u += kThreads * 2) {
            const float4 v = *reinterpret_cast<const float4 *>(buf + u);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int uu = u + h;
                const int a = ctl.decA[0][uu & 63] | ctl.decA[1][uu >> 6];
                const int m = ctl.decM[0][uu & 63] | ctl.decM[1][uu >> 6];
                const float re = h ? v.z : v.x, im = h ? v.w : v.y;
                const float rh = tf32_rna(re), ih = tf32_rna(im);
                const float rl = tf32_rna(re - rh), il = tf32_rna(im - ih);
                const int kk = 2 * a;
                const uint32_t off = uint32_t(kk >> 5) * C::A_CHUNK + uint32_t(m >> 3) * 1024 + uint32_t(m & 7) * 128 +
                                     uint32_t((((kk & 31) >> 2) ^ (m & 7)) << 4) + uint32_t((kk & 3) << 2);
                *reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(Ahi) + off) = make_float2(rh, ih);
                *reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(Alo) + off) = make_float2(rl, il);
            }
        }
        fence_proxy_async();
        __syncthreads();

        if (tid == 0) {
            tc_fence_after();
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
            const uint32_t As[3] = {al, ah, ah}, Bs[3] = {bh, bl, bh};  // small products first
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
#pragma unroll
                for (int ks = 0; ks < C::KR / 8; ++ks) {
                    const uint32_t koff = uint32_t(ks & 3) * 32;
                    const uint64_t ad = sw128_desc(As[pr] + uint32_t(ks >> 2) * C::A_CHUNK + koff);
                    const uint64_t bd = sw128_desc(Bs[pr] + uint32_t(ks >> 2) * C::B_CHUNK + koff);
                    mma_tf32(tmem, ad, bd, IDESC, (pr | ks) != 0);
                }
            }
            mma_commit(&ctl.bar_mma);
            // the store of tile i-1 must have read its buffer before tile i+2 lands in it
            bulk_wait_read_all();
            if (issued < n_local) issue_load(issued++);
        }
        ok = mbar_wait(&ctl.bar_mma, uint32_t(i & 1));
        if (__syncthreads_or(!ok)) { ok = false; break; }
        tc_fence_after();

        // epilogue: warp w reads TMEM lanes 32(w%4).. (rows m) and half the columns
        {
            const int m = 32 * (warp & 3) + lane;
            const int half = warp >> 2;
            const uint32_t taddr = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(half * (C::KR / 2));
            const uint32_t pm = ctl.posM[m];
            constexpr int NJ = C::KR / 4;  // amplitudes per thread
            float sx = 0.f;
            if (d.unitary) {
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const float2 x = buf[ctl.posA[half * NJ + j] | pm];
                    sx = fmaf(x.x, x.x, fmaf(x.y, x.y, sx));
                }
            }
            float v[2 * NJ];
            if constexpr (NJ == 16)
                tmem_ld32(taddr, v);
            else
                tmem_ld16(taddr, v);
            if (d.unitary) {
                float sy = 0.f;
#pragma unroll
                for (int j = 0; j < 2 * NJ; ++j) sy = fmaf(v[j], v[j], sy);
                ctl.red[half][m] = make_float2(sx, sy);
                __syncthreads();
                const float tx = ctl.red[0][m].x + ctl.red[1][m].x;
                const float ty = ctl.red[0][m].y + ctl.red[1][m].y;
                // sqrt(tx/ty) - 1 to first order, kept as a small number: the
                // bias is a fraction of an ulp, so a scale factor near 1 would
                // round to exactly 1; v + v c rounds to nearest, unbiased.
                const float c = (tx > 0.f && ty > 0.f) ? (tx - ty) / (2.f * ty) : 0.f;
#pragma unroll
                for (int j = 0; j < 2 * NJ; ++j) v[j] = fmaf(v[j], c, v[j]);
            }
#pragma unroll
            for (int j = 0; j < NJ; ++j) buf[ctl.posA[half * NJ + j] | pm] = make_float2(v[2 * j], v[2 * j + 1]);
        }
        tc_fence_before();
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            const uint64_t base = tile_base(i);
            for (int r = 0; r < nrun; ++r)
                bulk_s2g(dst + base + ctl.runoff[r], buf + size_t(r) * run_amps, run_amps * 8);
            bulk_commit();
        }
    }

    if (!ok) {
        if (tid == 0) atomicExch(status, QSIM_ETIMEOUT);
        ctl.abort = 1;
    }
    if (tid == 0) {
        // wait (bounded) for loads still in flight, then for the stores
        const uint64_t n_consumed = ok ? n_local : 0;
        for (uint64_t j = n_consumed; j < issued; ++j)
            if (j + kNBuf >= issued) mbar_wait(&ctl.bar_load[j % kNBuf], uint32_t((j / kNBuf) & 1));
        bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, C::TMEM_COLS);
}

}  // namespace

int fused_prepare() {
    static int configured[64];
    int dev = 0;
    QS_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && configured[dev]) return QSIM_OK;
    QS_CUDA(cudaFuncSetAttribute(k_fused_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg<4>::SMEM)));
    QS_CUDA(cudaFuncSetAttribute(k_fused_tc<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg<5>::SMEM)));
    if (dev < 64) configured[dev] = 1;
    return QSIM_OK;
}

size_t fused_rimg_floats(int k) { return 2 * size_t(4) << (2 * k); }  // 2 x (2^(k+1))^2

int launch_fused(void *dst, const void *src, int M, const FusedDesc &d, const float *rimg_dev, int *status,
                 cudaStream_t s) {
    if (int rc = fused_prepare()) return rc;
    const uint64_t ntiles = uint64_t(1) << (M - d.k - 7);
    const int per_sm = d.k == 4 ? 2 : 1;
    uint64_t grid = uint64_t(num_sms()) * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (d.k == 5)
        k_fused_tc<5><<<unsigned(grid), kThreads, Cfg<5>::SMEM, s>>>(
            static_cast<float2 *>(dst), static_cast<const float2 *>(src), d, rimg_dev, ntiles, status);
    else
        k_fused_tc<4><<<unsigned(grid), kThreads, Cfg<4>::SMEM, s>>>(
            static_cast<float2 *>(dst), static_cast<const float2 *>(src), d, rimg_dev, ntiles, status);
    QS_CHECK_LAUNCH("fused tensor-core launch");
    return QSIM_OK;
}

}  // namespace qs
