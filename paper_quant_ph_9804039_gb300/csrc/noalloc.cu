// Fidelity and norm with no device allocation at all.
//
// Some callers cannot allocate device memory: plugins inside a host
// application that hands out all of the GPU's memory from its own pool (a
// cudaMalloc of their own would fail or break the host's accounting), and
// latency-critical loops that must never enter the allocator, whose first
// call could otherwise stall on it.  qsim_fidelity needs a qsim_state, and
// creating one allocates the reduction's scratch; this file gives those
// callers the same reduction over plain device pointers they already own.
//
// The scratch (one partial sum per span of 2^16 amplitudes, plus the final
// result) lives in a fixed file-scope device array below: every GPU that
// loads the library holds it (1.5 MiB) until the process exits.  In host
// code the array's name is only a host-side stand-in, so its device address
// is looked up once per device with cudaGetSymbolAddress and passed to the
// kernels.  The address is kept for the life of the process: it assumes the
// device's primary context is not torn down (cudaDeviceReset) and re-created
// in between.
//
// The call reads its result back to the host and waits for its stream.
//
// Every call shares the one array.  Each call writes every partial slot it
// reads before reading it, so nothing has to start at zero, but two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on the array and may return each other's sums.
#include <mutex>

#include "cx.cuh"
#include "qsim_internal.h"

namespace {

constexpr int kSpanBits = 16;                                // amplitudes per partial sum: 2^16
constexpr int64_t kMaxSpans = int64_t(1) << 16;              // partial sums the array holds
constexpr int kMaxQubits = kSpanBits + 16;                   // so M <= 32
constexpr int64_t kResult = 3 * kMaxSpans;                   // index of (norm, re, im)

static __device__ __align__(256) double g_noalloc_scratch[3 * kMaxSpans + 4];

std::mutex g_setup_mu;
double *g_scratch_addr[64];  // device address of g_noalloc_scratch, per device

// Set-up, once per device, with that device current.
int scratch_address(double **out) {
    int dev = 0;
    QS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        qs::set_error("device index %d out of range", dev);
        return QSIM_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return qs::cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return QSIM_OK;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ void block_sum3(double &a, double &b, double &c) {
    __shared__ double sh[3][32];
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = a; sh[1][w] = b; sh[2][w] = c; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = warp_sum(l < nw ? sh[0][l] : 0.0);
        b = warp_sum(l < nw ? sh[1][l] : 0.0);
        c = warp_sum(l < nw ? sh[2][l] : 0.0);
    }
}

// Block s adds the amplitudes [s * 2^16, min(N, (s+1) * 2^16)): norm of the
// noisy vector and, when `id` is given, sum conj(id_i) nz_i.  complex64 values
// are multiplied and summed in float over groups of 8, then in double.
template <bool FID>
__global__ void __launch_bounds__(256) k_span_f(const float2 *__restrict__ id, const float2 *__restrict__ nz,
                                                uint64_t N, double *__restrict__ partials) {
    const uint64_t lo = uint64_t(blockIdx.x) << kSpanBits;
    const uint64_t hi = (lo + (uint64_t(1) << kSpanBits) < N) ? lo + (uint64_t(1) << kSpanBits) : N;
    double sn = 0.0, sre = 0.0, sim = 0.0;
    if (hi - lo >= 8) {
        const float4 *b4 = reinterpret_cast<const float4 *>(nz);
        const float4 *a4 = reinterpret_cast<const float4 *>(id);
        for (uint64_t g = lo / 8 + threadIdx.x; g < hi / 8; g += blockDim.x) {
            float fn = 0.f, fre = 0.f, fim = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 b = b4[g * 4 + k];
                fn = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, fmaf(b.w, b.w, fn))));
                if (FID) {
                    const float4 a = a4[g * 4 + k];
                    fre = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, fre))));
                    fim = fmaf(a.x, b.y, fmaf(-a.y, b.x, fmaf(a.z, b.w, fmaf(-a.w, b.z, fim))));
                }
            }
            sn += double(fn);
            sre += double(fre);
            sim += double(fim);
        }
    } else {
        for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double br = nz[i].x, bi = nz[i].y;
            sn += br * br + bi * bi;
            if (FID) {
                const double ar = id[i].x, ai = id[i].y;
                sre += ar * br + ai * bi;
                sim += ar * bi - ai * br;
            }
        }
    }
    block_sum3(sn, sre, sim);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = sn;
        partials[3 * blockIdx.x + 1] = sre;
        partials[3 * blockIdx.x + 2] = sim;
    }
}

template <bool FID>
__global__ void __launch_bounds__(256) k_span_d(const double2 *__restrict__ id, const double2 *__restrict__ nz,
                                                uint64_t N, double *__restrict__ partials) {
    const uint64_t lo = uint64_t(blockIdx.x) << kSpanBits;
    const uint64_t hi = (lo + (uint64_t(1) << kSpanBits) < N) ? lo + (uint64_t(1) << kSpanBits) : N;
    double sn = 0.0, sre = 0.0, sim = 0.0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double br = nz[i].x, bi = nz[i].y;
        sn = fma(br, br, fma(bi, bi, sn));
        if (FID) {
            const double ar = id[i].x, ai = id[i].y;
            sre = fma(ar, br, fma(ai, bi, sre));
            sim = fma(ar, bi, fma(-ai, br, sim));
        }
    }
    block_sum3(sn, sre, sim);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = sn;
        partials[3 * blockIdx.x + 1] = sre;
        partials[3 * blockIdx.x + 2] = sim;
    }
}

// Adds the nspans partial sums in a fixed order and stores the totals.
__global__ void __launch_bounds__(1024) k_span_total(double *scratch, int64_t nspans) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t j = threadIdx.x; j < nspans; j += blockDim.x) {
        a += scratch[3 * j + 0];
        b += scratch[3 * j + 1];
        c += scratch[3 * j + 2];
    }
    block_sum3(a, b, c);
    if (threadIdx.x == 0) {
        scratch[kResult + 0] = a;
        scratch[kResult + 1] = b;
        scratch[kResult + 2] = c;
    }
}

}  // namespace

extern "C" int qsim_fidelity_noalloc(const void *ideal_amps, const void *noisy_amps, int M, qsim_prec prec,
                                     void *cuda_stream, double *F, double *norm_noisy) {
    using namespace qs;
    if (M < 1 || M > kMaxQubits) {
        set_error("qsim_fidelity_noalloc: M = %d is outside [1, %d]; its fixed scratch holds %lld partial sums "
                  "of 2^%d amplitudes each (use qsim_fidelity for larger states)",
                  M, kMaxQubits, (long long)kMaxSpans, kSpanBits);
        return QSIM_EINVAL;
    }
    if (prec != QSIM_C64 && prec != QSIM_C128) {
        set_error("qsim_fidelity_noalloc: unknown precision %d", int(prec));
        return QSIM_EINVAL;
    }
    if (!noisy_amps || (reinterpret_cast<uintptr_t>(noisy_amps) & 15) ||
        (reinterpret_cast<uintptr_t>(ideal_amps) & 15)) {
        set_error("qsim_fidelity_noalloc: amplitudes must be non-NULL, 16-byte aligned device pointers");
        return QSIM_EINVAL;
    }
    const uint64_t N = uint64_t(1) << M;
    const int64_t nspans = int64_t((N + (uint64_t(1) << kSpanBits) - 1) >> kSpanBits);
    if (nspans > kMaxSpans) {  // unreachable while kMaxQubits is checked above; kept with the array size
        set_error("qsim_fidelity_noalloc: %lld partial sums needed, the fixed scratch holds %lld",
                  (long long)nspans, (long long)kMaxSpans);
        return QSIM_EINVAL;
    }
    double *scratch = nullptr;
    if (int rc = scratch_address(&scratch)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const bool fid = ideal_amps != nullptr;
    if (prec == QSIM_C64) {
        const float2 *a = static_cast<const float2 *>(ideal_amps), *b = static_cast<const float2 *>(noisy_amps);
        if (fid) k_span_f<true><<<unsigned(nspans), 256, 0, s>>>(a, b, N, scratch);
        else k_span_f<false><<<unsigned(nspans), 256, 0, s>>>(nullptr, b, N, scratch);
    } else {
        const double2 *a = static_cast<const double2 *>(ideal_amps), *b = static_cast<const double2 *>(noisy_amps);
        if (fid) k_span_d<true><<<unsigned(nspans), 256, 0, s>>>(a, b, N, scratch);
        else k_span_d<false><<<unsigned(nspans), 256, 0, s>>>(nullptr, b, N, scratch);
    }
    QS_CHECK_LAUNCH("no-allocation reduction launch");
    k_span_total<<<1, 1024, 0, s>>>(scratch, nspans);
    QS_CHECK_LAUNCH("no-allocation total launch");
    double r[3];
    QS_CUDA(cudaMemcpyAsync(r, scratch + kResult, sizeof(r), cudaMemcpyDeviceToHost, s));
    QS_CUDA(cudaStreamSynchronize(s));
    if (F) *F = fid ? r[1] * r[1] + r[2] * r[2] : 0.0;
    if (norm_noisy) *norm_noisy = r[0];
    return QSIM_OK;
}
