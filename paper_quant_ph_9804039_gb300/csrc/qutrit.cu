// The three-state model (Section 2.0; Sections 3.0-3.1): M three-level
// particles, 3^M complex amplitudes, the index written in base 3 with digit q
// the level of particle q (digit 0 least significant).  A transformation on
// particle t is a 3x3 matrix U applied to every triple of states that differ
// only in that particle's level, (a_i, a_{i + 3^t}, a_{i + 2 3^t}) for every i
// whose digit t is 0 (the three-state form of Figure 3); a control (c, v)
// restricts it to the triples whose digit c is v.
//
// One launch per transformation, one thread per triple (grid-stride): the
// triple index k = hi 3^t + lo maps to i = hi 3^(t+1) + lo, so consecutive
// threads read consecutive amplitudes of each of the three slices (for
// t = 0, three consecutive amplitudes each).  The divisions by powers of three
// go through a 64-bit multiply-high with a one-step correction (div_pow3,
// exact for the indices used, below 2^40).  Triples whose controls are not at their levels
// are neither read nor written.  complex64 uses the compensated (hi + lo)
// matrix entries of the other kernels.
#include <cmath>

#include "cx.cuh"
#include "qsim_internal.h"

namespace qs {
namespace {

constexpr int kMaxQutrits = 21;  // 3^21 complex64 amplitudes = 84 GB

template <typename T2>
struct Gate3K {
    T2 uh[9], ul[9];
    uint64_t st;            // 3^t
    uint64_t mst;           // its division multiplier (div_magic)
    int nc;
    uint64_t cpw[2];        // 3^c of each control
    uint64_t cm[2];
    int lvl[2];
};

// Division by d > 1 through a 64-bit multiply-high: with m = floor(2^64 / d) + 1
// (d not a power of two), q = mulhi(x, m) is floor(x / d) or one more, for
// x < 2^40; one compare corrects it.  Integer pipes only (FP64 is slow here).
__host__ uint64_t div_magic(uint64_t d) { return d > 1 ? ~uint64_t(0) / d + 1 : 0; }
__device__ __forceinline__ uint64_t div_pow3(uint64_t x, uint64_t d, uint64_t m) {
    if (d == 1) return x;
    uint64_t q = __umul64hi(x, m);
    if (q * d > x) --q;
    return q;
}

template <typename T2>
__global__ void __launch_bounds__(256) k_gate3(T2 *__restrict__ a, uint64_t units, Gate3K<T2> g) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t k = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < units; k += stride) {
        const uint64_t hi = div_pow3(k, g.st, g.mst);
        const uint64_t i = hi * 3 * g.st + (k - hi * g.st);
        bool on = true;
        for (int c = 0; c < g.nc; ++c) {
            const uint64_t q = div_pow3(i, g.cpw[c], g.cm[c]);
            on = on && int(q % 3) == g.lvl[c];
        }
        if (!on) continue;
        const T2 x0 = a[i], x1 = a[i + g.st], x2 = a[i + 2 * g.st];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            T2 y = cmad2x(g.uh[3 * r], g.ul[3 * r], x0, g.uh[3 * r + 1], g.ul[3 * r + 1], x1);
            const T2 z = cmulx(g.uh[3 * r + 2], g.ul[3 * r + 2], x2);
            y.x += z.x;
            y.y += z.y;
            a[i + uint64_t(r) * g.st] = y;
        }
    }
}

constexpr int kSpan = 1 << 16;

// Block s sums the amplitudes [s kSpan, min(n, (s+1) kSpan)): the norm of nz
// and, with id, sum conj(id_i) nz_i; a second kernel adds the blocks' sums in
// order.
template <typename T2>
__global__ void __launch_bounds__(256) k_sum3(const T2 *__restrict__ id, const T2 *__restrict__ nz, uint64_t n,
                                              double *__restrict__ part) {
    __shared__ double sh[3][8];
    const uint64_t lo = uint64_t(blockIdx.x) * kSpan, hi = lo + kSpan < n ? lo + kSpan : n;
    double sn = 0, sre = 0, sim = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double br = nz[i].x, bi = nz[i].y;
        sn += br * br + bi * bi;
        if (id) {
            const double ar = id[i].x, ai = id[i].y;
            sre += ar * br + ai * bi;
            sim += ar * bi - ai * br;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sn += __shfl_xor_sync(0xffffffffu, sn, o);
        sre += __shfl_xor_sync(0xffffffffu, sre, o);
        sim += __shfl_xor_sync(0xffffffffu, sim, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = sn;
        sh[1][w] = sre;
        sh[2][w] = sim;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int k = 0; k < int(blockDim.x >> 5); ++k) {
            a += sh[0][k];
            b += sh[1][k];
            c += sh[2][k];
        }
        part[3 * blockIdx.x] = a;
        part[3 * blockIdx.x + 1] = b;
        part[3 * blockIdx.x + 2] = c;
    }
}

__global__ void k_sum3_total(double *part, int64_t nblocks, double *out) {
    if (threadIdx.x != 0) return;
    double a = 0, b = 0, c = 0;
    for (int64_t j = 0; j < nblocks; ++j) {
        a += part[3 * j];
        b += part[3 * j + 1];
        c += part[3 * j + 2];
    }
    out[0] = a;
    out[1] = b;
    out[2] = c;
}

uint64_t pow3(int k) {
    uint64_t v = 1;
    for (int i = 0; i < k; ++i) v *= 3;
    return v;
}

int check3(int M, qsim_prec prec, const void *amps) {
    if (M < 1 || M > kMaxQutrits) {
        set_error("M = %d outside [1, %d] particles", M, kMaxQutrits);
        return QSIM_EINVAL;
    }
    if (prec != QSIM_C64 && prec != QSIM_C128) {
        set_error("unknown precision %d", int(prec));
        return QSIM_EINVAL;
    }
    if (!amps || (reinterpret_cast<uintptr_t>(amps) & 15)) {
        set_error("amplitudes must be a non-NULL, 16-byte aligned device pointer");
        return QSIM_EINVAL;
    }
    return QSIM_OK;
}

template <typename T2>
int apply(void *amps, int M, const qsim_gate3 *gates, size_t n, cudaStream_t s) {
    using R = decltype(T2{}.x);
    const uint64_t units = pow3(M - 1);
    const unsigned grid = unsigned(std::min<uint64_t>((units + 255) / 256, uint64_t(num_sms()) * 16));
    for (size_t gi = 0; gi < n; ++gi) {
        const qsim_gate3 &x = gates[gi];
        Gate3K<T2> g{};
        for (int e = 0; e < 9; ++e) {
            if (sizeof(R) == 4) {
                float hr, lr, hi, li;
                split_f(x.U[2 * e], hr, lr);
                split_f(x.U[2 * e + 1], hi, li);
                g.uh[e] = mk(R(hr), R(hi));
                g.ul[e] = mk(R(lr), R(li));
            } else {
                g.uh[e] = mk(R(x.U[2 * e]), R(x.U[2 * e + 1]));
                g.ul[e] = mk(R(0), R(0));
            }
        }
        g.st = pow3(x.target);
        g.mst = div_magic(g.st);
        g.nc = x.ncontrols;
        for (int c = 0; c < x.ncontrols; ++c) {
            g.cpw[c] = pow3(x.controls[c]);
            g.cm[c] = div_magic(g.cpw[c]);
            g.lvl[c] = x.levels[c];
        }
        k_gate3<T2><<<grid, 256, 0, s>>>(static_cast<T2 *>(amps), units, g);
        QS_CHECK_LAUNCH("qutrit transformation launch");
    }
    return QSIM_OK;
}

}  // namespace
}  // namespace qs

extern "C" int qsim_qutrit_apply(void *device_amps, int M, qsim_prec prec, const qsim_gate3 *gates, size_t n,
                                 void *cuda_stream) {
    using namespace qs;
    if (int rc = check3(M, prec, device_amps)) return rc;
    if (n > 0 && !gates) { set_error("gates is NULL"); return QSIM_EINVAL; }
    for (size_t i = 0; i < n; ++i) {
        const qsim_gate3 &g = gates[i];
        if (g.target < 0 || g.target >= M || g.ncontrols < 0 || g.ncontrols > 2) {
            set_error("transformation %zu: target %d or %d controls out of range", i, g.target, g.ncontrols);
            return QSIM_EINVAL;
        }
        for (int c = 0; c < g.ncontrols; ++c)
            if (g.controls[c] < 0 || g.controls[c] >= M || g.controls[c] == g.target || g.levels[c] < 0 ||
                g.levels[c] > 2 || (c == 1 && g.controls[1] == g.controls[0])) {
                set_error("transformation %zu: bad control %d (level %d)", i, g.controls[c], g.levels[c]);
                return QSIM_EINVAL;
            }
        for (int e = 0; e < 18; ++e)
            if (!std::isfinite(g.U[e])) { set_error("transformation %zu: matrix not finite", i); return QSIM_EINVAL; }
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    return prec == QSIM_C64 ? apply<float2>(device_amps, M, gates, n, s) : apply<double2>(device_amps, M, gates, n, s);
}

extern "C" int qsim_qutrit_overlap(const void *ideal_amps, const void *noisy_amps, int M, qsim_prec prec,
                                   void *cuda_stream, double out[3]) {
    using namespace qs;
    if (int rc = check3(M, prec, noisy_amps)) return rc;
    if (!out) { set_error("out is NULL"); return QSIM_EINVAL; }
    if (reinterpret_cast<uintptr_t>(ideal_amps) & 15) { set_error("ideal amplitudes not 16-byte aligned"); return QSIM_EINVAL; }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const uint64_t n = pow3(M);
    const int64_t nb = int64_t((n + kSpan - 1) / kSpan);
    const DevAllocator al = current_allocator();
    void *buf = nullptr;
    const size_t bytes = (3 * size_t(nb) + 3) * sizeof(double);
    if (int rc = dmalloc(al, &buf, bytes, s, "qutrit sums")) return rc;
    double *part = static_cast<double *>(buf);
    int rc = QSIM_OK;
    if (prec == QSIM_C64)
        k_sum3<float2><<<unsigned(nb), 256, 0, s>>>(static_cast<const float2 *>(ideal_amps),
                                                    static_cast<const float2 *>(noisy_amps), n, part);
    else
        k_sum3<double2><<<unsigned(nb), 256, 0, s>>>(static_cast<const double2 *>(ideal_amps),
                                                     static_cast<const double2 *>(noisy_amps), n, part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_sum3_total<<<1, 32, 0, s>>>(part, nb, part + 3 * nb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, part + 3 * nb, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "qutrit sums");
    dfree(al, buf, bytes, s);
    return rc;
}
