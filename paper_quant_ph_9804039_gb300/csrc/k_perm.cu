// Qubit permutation pass: the state after a run of SWAP gates (each three
// exact CNOTs, Section 1.3 Table 1 / Figure 2) whose composition pi is an
// involution on qubit positions (disjoint swaps, e.g. the bit reversal that
// ends the quantum FFT).  out[pi(i)] = in[i], where pi moves bit q of the
// index to bit pi(q): one read and one write of the vector instead of one
// pass per CNOT, with no arithmetic (bit-exact).
//
// Tiles hold the qubits S = {0..lb-1} u pi({0..lb-1}); pi maps S onto itself
// and the other qubits onto each other, so tile o (outside bits o) maps onto
// tile pi(o).  A block reads tile o and its partner, both as runs of 2^lb
// contiguous amplitudes (every thread's loads of both tiles in flight at
// once), and writes each into the other's place, reading shared memory in the
// permuted order.  Shared memory holds amplitude u at u ^ ((u >> sh) & 15),
// with the shift picked on the host so that both the writes in index order
// and the permuted reads of a warp fall on distinct banks.  In place is safe:
// a pair is read completely before it is written.
#include "qsim_internal.h"

namespace qs {
namespace {

constexpr int kPermThreads = 256;

// One amplitude global -> shared, asynchronously (cp.async; 8 or 16 bytes).
__device__ __forceinline__ void cp_async_amp(float2 *dst, const float2 *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_amp(double2 *dst, const double2 *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }


// The first lb tile qubits are qubits 0..lb-1, so a local index u sits at
// offset (u & (2^lb - 1)) | hoff[u >> lb] of the vector; sig(u) (the local
// index whose amplitude lands on u) splits the same way over the two parts.
template <typename T2>
__global__ void __launch_bounds__(kPermThreads) k_permute(T2 *dst, const T2 *src, PermDesc d, uint64_t ntiles) {

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ns = d.ns, lb = d.lb;
    const uint32_t n = 1u << ns, lmask = (1u << lb) - 1, nh = n >> lb;
    T2 *A = reinterpret_cast<T2 *>(smem_raw);
    T2 *B = A + n;
    uint64_t *hoff = reinterpret_cast<uint64_t *>(B + n);  // high local bits -> offset bits
    uint32_t *slo = reinterpret_cast<uint32_t *>(hoff + nh);  // sig of the low / high local bits
    uint32_t *shi = slo + (lmask + 1);
    for (uint32_t u = threadIdx.x; u <= lmask || u < nh; u += blockDim.x) {
        if (u <= lmask) {
            uint32_t v = 0;
            for (int j = 0; j < lb; ++j)
                if ((u >> j) & 1) v |= 1u << d.spi[j];
            slo[u] = v;
        }
        if (u < nh) {
            uint32_t v = 0;
            uint64_t off = 0;
            for (int j = lb; j < ns; ++j)
                if ((u >> (j - lb)) & 1) {
                    v |= 1u << d.spi[j];
                    off |= uint64_t(1) << d.spos[j];
                }
            shi[u] = v;
            hoff[u] = off;
        }
    }
    __syncthreads();
    const int sh = d.sh;
    auto pad = [sh](uint32_t u) { return u ^ ((u >> sh) & 15u); };
    for (uint64_t o = blockIdx.x; o < ntiles; o += gridDim.x) {
        uint64_t o2 = 0, base = 0, base2 = 0;
        for (int j = 0; j < d.nout; ++j)
            if ((o >> j) & 1) {
                o2 |= uint64_t(1) << d.opi[j];
                base |= uint64_t(1) << d.opos[j];
                base2 |= uint64_t(1) << d.opos[d.opi[j]];
            }
        if (o2 < o) continue;  // the partner's block does this pair
        // asynchronous copies straight into shared memory: every load of the
        // block in flight at once, no registers held
        if (o2 != o) {
            for (uint32_t u = threadIdx.x; u < n; u += kPermThreads) {
                const uint64_t off = (u & lmask) | hoff[u >> lb];
                cp_async_amp(A + pad(u), src + (base | off));
                cp_async_amp(B + pad(u), src + (base2 | off));
            }
            cp_async_wait();
            __syncthreads();
            // tile o lands on tile o2: out[base2 | off(v)] = A[sig^-1(v)] = A[sig(v)]
            for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
                const uint32_t ps = pad(slo[v & lmask] | shi[v >> lb]);
                const uint64_t off = (v & lmask) | hoff[v >> lb];
                dst[base2 | off] = A[ps];
                dst[base | off] = B[ps];
            }
        } else {
            for (uint32_t u = threadIdx.x; u < n; u += kPermThreads)
                cp_async_amp(A + pad(u), src + (base | (u & lmask) | hoff[u >> lb]));
            cp_async_wait();
            __syncthreads();
            for (uint32_t v = threadIdx.x; v < n; v += blockDim.x)
                dst[base | (v & lmask) | hoff[v >> lb]] = A[pad(slo[v & lmask] | shi[v >> lb])];
        }
        __syncthreads();
    }
}

template <typename T2>
size_t perm_smem(const PermDesc &d) {
    const size_t n = size_t(1) << d.ns, nh = n >> d.lb, nl = size_t(1) << d.lb;
    return 2 * n * sizeof(T2) + nh * sizeof(uint64_t) + (nl + nh) * sizeof(uint32_t);
}

template <typename T2>
int launch_t(T2 *dst, const T2 *src, const PermDesc &d, cudaStream_t s) {
    const uint64_t ntiles = uint64_t(1) << d.nout;
    const size_t smem = perm_smem<T2>(d);
    static int configured[64];
    int dev = 0;
    QS_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !configured[dev]) {
        QS_CUDA(cudaFuncSetAttribute(k_permute<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        configured[dev] = 1;
    }
    int per_sm = 0;
    QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_permute<T2>, kPermThreads, smem));
    uint64_t grid = uint64_t(num_sms()) * uint64_t(per_sm < 1 ? 1 : per_sm);
    if (grid > ntiles) grid = ntiles;
    k_permute<T2><<<unsigned(grid), kPermThreads, smem, s>>>(dst, src, d, ntiles);
    QS_CHECK_LAUNCH("permutation launch");
    return QSIM_OK;
}

}  // namespace

size_t perm_smem_bytes(const PermDesc &d, qsim_prec prec) {
    return prec == QSIM_C64 ? perm_smem<float2>(d) : perm_smem<double2>(d);
}

int launch_perm(void *dst, const void *src, int M, qsim_prec prec, const PermDesc &d, cudaStream_t s) {
    (void)M;
    if (prec == QSIM_C64)
        return launch_t(static_cast<float2 *>(dst), static_cast<const float2 *>(src), d, s);
    return launch_t(static_cast<double2 *>(dst), static_cast<const double2 *>(src), d, s);
}

}  // namespace qs
