// Reductions over the state vector and the |0...0> initialiser.
//
//   k_reduce       norm = sum |n_i|^2 (Section 1.2: the probabilities of all
//                  states sum to one) and, with a second vector, the overlap
//                  sum conj(id_i) n_i from which F = |<ideal|noisy>|^2.  Each
//                  thread adds 8 products in float32 (the products of two
//                  complex64 values need no more), then accumulates those
//                  partial sums in float64; warp shuffles and one shared-memory
//                  step reduce a block to one partial per block.
//   k_reduce_final one block adds the per-block partials in a fixed order, so
//                  the result is the same on every run.
//   k_probs        p_i = |a_i|^2 (Section 1.2, Figure 1).
#include "cx.cuh"
#include "qsim_internal.h"

namespace qs {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of three doubles; thread 0 gets the totals.
__device__ __forceinline__ void block_sum3(double &a, double &b, double &c) {
    __shared__ double sh[3][32];
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = a; sh[1][w] = b; sh[2][w] = c; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = l < nw ? sh[0][l] : 0.0;
        b = l < nw ? sh[1][l] : 0.0;
        c = l < nw ? sh[2][l] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
    }
}

// complex64: 8 amplitudes (four 16-byte loads per vector) per iteration.
template <bool FID>
__global__ void __launch_bounds__(256) k_reduce_f(const float4 *__restrict__ id, const float4 *__restrict__ nz,
                                                  uint64_t ngroups, double *__restrict__ partials) {
    double sn = 0.0, sre = 0.0, sim = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t gi = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; gi < ngroups; gi += stride) {
        float4 b[4], a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) b[k] = __ldcs(nz + gi * 4 + k);
        if (FID) {
#pragma unroll
            for (int k = 0; k < 4; ++k) a[k] = __ldcs(id + gi * 4 + k);
        }
        float fn = 0.f, fre = 0.f, fim = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            fn = fmaf(b[k].x, b[k].x, fn);
            fn = fmaf(b[k].y, b[k].y, fn);
            fn = fmaf(b[k].z, b[k].z, fn);
            fn = fmaf(b[k].w, b[k].w, fn);
            if (FID) {  // conj(a) * b = (ar br + ai bi) + i (ar bi - ai br)
                fre = fmaf(a[k].x, b[k].x, fre);
                fre = fmaf(a[k].y, b[k].y, fre);
                fre = fmaf(a[k].z, b[k].z, fre);
                fre = fmaf(a[k].w, b[k].w, fre);
                fim = fmaf(a[k].x, b[k].y, fim);
                fim = fmaf(-a[k].y, b[k].x, fim);
                fim = fmaf(a[k].z, b[k].w, fim);
                fim = fmaf(-a[k].w, b[k].z, fim);
            }
        }
        sn += double(fn);
        sre += double(fre);
        sim += double(fim);
    }
    block_sum3(sn, sre, sim);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = sn;
        partials[3 * blockIdx.x + 1] = sre;
        partials[3 * blockIdx.x + 2] = sim;
    }
}

// complex128 (and the tail of small complex64 vectors): one amplitude per step,
// all in double.
template <typename T2, bool FID>
__global__ void __launch_bounds__(256) k_reduce_scalar(const T2 *__restrict__ id, const T2 *__restrict__ nz,
                                                       uint64_t n, double *__restrict__ partials) {
    double sn = 0.0, sre = 0.0, sim = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
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

__global__ void __launch_bounds__(1024) k_reduce_final(const double *__restrict__ partials, int nparts,
                                                       double *__restrict__ out) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int j = threadIdx.x; j < nparts; j += blockDim.x) {
        a += partials[3 * j + 0];
        b += partials[3 * j + 1];
        c += partials[3 * j + 2];
    }
    block_sum3(a, b, c);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
        out[2] = c;
    }
}

__global__ void k_probs_f(const float4 *__restrict__ a, float2 *__restrict__ p, uint64_t nvec) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nvec;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const float4 v = a[i];
        p[i] = make_float2(fmaf(v.x, v.x, v.y * v.y), fmaf(v.z, v.z, v.w * v.w));
    }
}

template <typename T2, typename P>
__global__ void k_probs_scalar(const T2 *__restrict__ a, P *__restrict__ p, uint64_t n) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const T2 v = a[i];
        p[i] = P(v.x) * P(v.x) + P(v.y) * P(v.y);
    }
}

template <typename T2>
__global__ void k_set_one(T2 *a) {
    a[0].x = 1;
    a[0].y = 0;
}

unsigned grid_cap(uint64_t items, int per_block, uint64_t cap) {
    uint64_t g = (items + per_block - 1) / per_block;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return unsigned(g);
}

}  // namespace

int launch_reduce(const void *ideal, const void *noisy, int M, qsim_prec prec, double *scratch,
                  int scratch_blocks, cudaStream_t s) {
    const uint64_t N = uint64_t(1) << M;
    const bool fid = ideal != nullptr;
    uint64_t cap = uint64_t(num_sms()) * 8;
    if (cap > uint64_t(scratch_blocks)) cap = uint64_t(scratch_blocks);
    double *out = scratch + 3 * size_t(scratch_blocks);
    unsigned grid;
    if (prec == QSIM_C64 && N >= 8) {
        const uint64_t ngroups = N / 8;
        grid = grid_cap(ngroups, 256, cap);
        if (fid)
            k_reduce_f<true><<<grid, 256, 0, s>>>(static_cast<const float4 *>(ideal),
                                                  static_cast<const float4 *>(noisy), ngroups, scratch);
        else
            k_reduce_f<false><<<grid, 256, 0, s>>>(nullptr, static_cast<const float4 *>(noisy), ngroups, scratch);
    } else if (prec == QSIM_C64) {
        grid = 1;
        if (fid)
            k_reduce_scalar<float2, true><<<1, 256, 0, s>>>(static_cast<const float2 *>(ideal),
                                                            static_cast<const float2 *>(noisy), N, scratch);
        else
            k_reduce_scalar<float2, false><<<1, 256, 0, s>>>(nullptr, static_cast<const float2 *>(noisy), N, scratch);
    } else {
        grid = grid_cap(N, 256, cap);
        if (fid)
            k_reduce_scalar<double2, true><<<grid, 256, 0, s>>>(static_cast<const double2 *>(ideal),
                                                                static_cast<const double2 *>(noisy), N, scratch);
        else
            k_reduce_scalar<double2, false><<<grid, 256, 0, s>>>(nullptr, static_cast<const double2 *>(noisy), N,
                                                                 scratch);
    }
    QS_CHECK_LAUNCH("reduction launch");
    k_reduce_final<<<1, 1024, 0, s>>>(scratch, int(grid), out);
    QS_CHECK_LAUNCH("final reduction launch");
    return QSIM_OK;
}

int launch_probabilities(const void *amps, int M, qsim_prec prec, void *out, cudaStream_t s) {
    const uint64_t N = uint64_t(1) << M;
    const uint64_t cap = uint64_t(num_sms()) * 16;
    if (prec == QSIM_C64 && N >= 2) {
        k_probs_f<<<grid_cap(N / 2, 256, cap), 256, 0, s>>>(static_cast<const float4 *>(amps),
                                                             static_cast<float2 *>(out), N / 2);
    } else if (prec == QSIM_C64) {
        k_probs_scalar<float2, float><<<1, 32, 0, s>>>(static_cast<const float2 *>(amps), static_cast<float *>(out), N);
    } else {
        k_probs_scalar<double2, double><<<grid_cap(N, 256, cap), 256, 0, s>>>(
            static_cast<const double2 *>(amps), static_cast<double *>(out), N);
    }
    QS_CHECK_LAUNCH("probabilities launch");
    return QSIM_OK;
}

int launch_zero_state(void *amps, int M, qsim_prec prec, cudaStream_t s) {
    QS_CUDA(cudaMemsetAsync(amps, 0, (size_t(1) << M) * amp_bytes(prec), s));
    if (prec == QSIM_C64)
        k_set_one<float2><<<1, 1, 0, s>>>(static_cast<float2 *>(amps));
    else
        k_set_one<double2><<<1, 1, 0, s>>>(static_cast<double2 *>(amps));
    QS_CHECK_LAUNCH("zero-state launch");
    return QSIM_OK;
}

}  // namespace qs
