// Decoherence after every operation (Section 3.4: two more transformations
// after each operation and a sum over the whole state; EQ 3, EQ 8).  The
// paper leaves the transformations open; the reading taken (and written out
// in the oracle): after gate g on target t,
//   1. a dephasing kick Rz(delta_g) on t (a diagonal unitary, no sum);
//   2. amplitude damping on t as a quantum jump: with P1 the weight of t's 1
//      states and N the norm, the jump probability is p = gamma P1 / N; for
//      r_g < p the jump operator [[0, sqrt gamma], [0, 0]], else the no-jump
//      operator diag(1, sqrt(1 - gamma)), each scaled to keep the norm N.
//
// The decision of operation g needs the whole state's sums after it, so one
// operation cannot share a pass with the next; but it can share the pass
// that applies the next gate.  One launch per operation: every block first
// adds up the previous launch's per-block sums (the same fixed order in every
// block, so all blocks take the same decision), builds that operation's
// damping matrix in FP64, applies it on the previous target and then this
// operation's gate (with its dephasing folded in, Rz(delta) U) on this
// target -- on quadruples of amplitudes when the targets differ, on pairs when
// they are the same -- and writes its own sums of P1 and N for the next
// launch.  A last launch applies the last damping.  Each operation costs one
// pass over the vector (16 bytes per amplitude for complex64) instead of the
// paper's three transformations plus a separate sum.
#include <cmath>

#include "cx.cuh"
#include "qsim_internal.h"

namespace qs {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxParts = 1024;

struct DecohOp {
    int tp;          // target of the previous operation's damping, -1 for none
    int t;           // target of this operation's gate, -1 for none (the last launch)
    uint64_t cmask;  // this gate's controls
    double U[8];     // Rz(delta) . U, row-major re/im
    double rz[2];    // cos(delta / 2), sin(delta / 2): the dephasing alone, where a control is 0
    double gamma;
    double r_prev;   // the previous operation's uniform draw
    int idx_prev;    // index of the previous operation (jumps / p outputs)
    int nparts;      // per-block sums written by the previous launch
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum of two values (every block gets the same result for
// the same inputs).
__device__ void block_sum2(double &a, double &b, double (*sh)[kThreads / 32]) {
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
    }
    __syncthreads();
    a = 0.0;
    b = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) {
        a += sh[0][k];
        b += sh[1][k];
    }
}

// v * (hi + lo): a real factor carried as two values of the state precision
template <typename T2, typename R>
__device__ __forceinline__ void scale2(T2 &v, R hi, R lo) {
    v.x = fma(v.x, hi, v.x * lo);
    v.y = fma(v.y, hi, v.y * lo);
}

// |v|^2 in the state precision
template <typename T2>
__device__ __forceinline__ auto weight(const T2 &v) -> decltype(v.x) {
    return fma(v.x, v.x, v.y * v.y);
}

// A running sum of weights.  complex64: a compensated (Kahan) float sum, so
// the loop issues no FP64 instruction at all (FP64 is a narrow pipe on this
// GPU: an earlier form that added a float group into a double every 8
// iterations kept the FP64 pipe 58 % busy and bounded the pass); the
// per-thread totals are then added in double.  complex128: double.
template <typename R>
struct WSum {
    R s = R(0), c = R(0);
    __device__ __forceinline__ void add(R v) {
        if (sizeof(R) == 8) {
            s += v;
        } else {
            const R y = v - c;
            const R t = s + y;
            c = (t - s) - y;
            s = t;
        }
    }
    __device__ __forceinline__ void next() {}
    __device__ __forceinline__ double total() const { return double(s) - double(c); }
};

template <typename T2>
__global__ void __launch_bounds__(kThreads) k_decoh(T2 *__restrict__ a, int M, DecohOp op,
                                                    const double *__restrict__ prev, double *__restrict__ part,
                                                    int *__restrict__ jumps, double *__restrict__ p_out) {
    using R = decltype(a[0].x);
    __shared__ double sh[2][kThreads / 32];
    __shared__ double kmat[3];  // jump: (0, c); no jump: (s0, s1); kmat[2] = 1 for a jump
    if (op.tp >= 0) {
        double P1 = 0.0, N = 0.0;
        for (int j = threadIdx.x; j < op.nparts; j += kThreads) {
            P1 += prev[2 * j];
            N += prev[2 * j + 1];
        }
        block_sum2(P1, N, sh);
        if (threadIdx.x == 0) {
            const double g = op.gamma;
            const double p = N > 0.0 ? g * P1 / N : 0.0;
            const bool jump = op.r_prev < p;
            if (jump) {
                kmat[0] = 0.0;
                kmat[1] = sqrt(g) * sqrt(N / (g * P1));
                kmat[2] = 1.0;
            } else {
                const double s = sqrt(N / (N - g * P1));
                kmat[0] = s;
                kmat[1] = sqrt(1.0 - g) * s;
                kmat[2] = 0.0;
            }
            if (blockIdx.x == 0) {
                jumps[op.idx_prev] = jump ? 1 : 0;
                p_out[op.idx_prev] = p;
            }
        }
        __syncthreads();
    }
    const bool has_k = op.tp >= 0, has_u = op.t >= 0;
    const bool kjump = has_k && kmat[2] != 0.0;
    const double k0 = has_k ? kmat[0] : 1.0, k1 = has_k ? kmat[1] : 1.0;
    const R k0h = R(k0), k0l = R(k0 - double(k0h)), k1h = R(k1), k1l = R(k1 - double(k1h));
    T2 uh[4], ul[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        R hr, lr, hi, li;
        if (sizeof(R) == 4) {
            float a0, b0, a1, b1;
            split_f(op.U[2 * e], a0, b0);
            split_f(op.U[2 * e + 1], a1, b1);
            hr = R(a0); lr = R(b0); hi = R(a1); li = R(b1);
        } else {
            hr = R(op.U[2 * e]); hi = R(op.U[2 * e + 1]); lr = R(0); li = R(0);
        }
        uh[e] = mk(hr, hi);
        ul[e] = mk(lr, li);
    }
    T2 rz_h[2], rz_l[2];  // Rz(delta): e^{-i delta/2}, e^{+i delta/2}
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const double re = op.rz[0], im = e ? op.rz[1] : -op.rz[1];
        if (sizeof(R) == 4) {
            float a0, b0, a1, b1;
            split_f(re, a0, b0);
            split_f(im, a1, b1);
            rz_h[e] = mk(R(a0), R(a1));
            rz_l[e] = mk(R(b0), R(b1));
        } else {
            rz_h[e] = mk(R(re), R(im));
            rz_l[e] = mk(R(0), R(0));
        }
    }
    // damping on one pair (lo: bit tp = 0, hi: bit tp = 1)
    auto damp = [&](T2 &lo, T2 &hi) {
        if (kjump) {
            lo = hi;
            scale2(lo, k1h, k1l);
            hi = mk(R(0), R(0));
        } else {
            scale2(lo, k0h, k0l);
            scale2(hi, k1h, k1l);
        }
    };
    // the gate and its dephasing on one pair (lo: bit t = 0); where a control
    // is 0 the dephasing alone
    auto gate = [&](uint64_t ilo, T2 &lo, T2 &hi) {
        if ((ilo & op.cmask) != op.cmask) {
            lo = cmulx(rz_h[0], rz_l[0], lo);
            hi = cmulx(rz_h[1], rz_l[1], hi);
            return;
        }
        const T2 x = lo, y = hi;
        lo = cmad2x(uh[0], ul[0], x, uh[1], ul[1], y);
        hi = cmad2x(uh[2], ul[2], x, uh[3], ul[3], y);
    };
    WSum<R> wP1, wN;
    const uint64_t stride = uint64_t(gridDim.x) * kThreads;
    if (has_k && has_u && op.tp != op.t) {
        const int lo_b = min(op.tp, op.t), hi_b = max(op.tp, op.t);
        const uint64_t bp = uint64_t(1) << op.tp, bt = uint64_t(1) << op.t;
        const uint64_t units = uint64_t(1) << (M - 2);
        for (uint64_t k = uint64_t(blockIdx.x) * kThreads + threadIdx.x; k < units; k += stride) {
            const uint64_t i = insert0(insert0(k, lo_b), hi_b);
            T2 v00 = a[i], v01 = a[i | bt], v10 = a[i | bp], v11 = a[i | bp | bt];  // v<tp bit><t bit>
            damp(v00, v10);
            damp(v01, v11);
            gate(i, v00, v01);
            gate(i | bp, v10, v11);
            a[i] = v00;
            a[i | bt] = v01;
            a[i | bp] = v10;
            a[i | bp | bt] = v11;
            const R w01 = weight(v01), w11 = weight(v11);
            wP1.add(w01 + w11);
            wN.add((weight(v00) + weight(v10)) + (w01 + w11));
            wP1.next();
            wN.next();
        }
    } else if (has_k || has_u) {
        const int b = has_u ? op.t : op.tp;
        const uint64_t bb = uint64_t(1) << b;
        const uint64_t units = uint64_t(1) << (M - 1);
        for (uint64_t k = uint64_t(blockIdx.x) * kThreads + threadIdx.x; k < units; k += stride) {
            const uint64_t i = insert0(k, b);
            T2 v0 = a[i], v1 = a[i | bb];
            if (has_k) damp(v0, v1);
            if (has_u) gate(i, v0, v1);
            a[i] = v0;
            a[i | bb] = v1;
            const R w1 = weight(v1);
            wP1.add(w1);
            wN.add(weight(v0) + w1);
            wP1.next();
            wN.next();
        }
    }
    double sP1 = wP1.total(), sN = wN.total();
    block_sum2(sP1, sN, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sP1;
        part[2 * blockIdx.x + 1] = sN;
    }
}

template <typename T2>
int run(qsim_state *st, const std::vector<Gate> &g, const double *delta, const double *r, double gamma, int *d_jumps,
        double *d_p, double *d_parts) {
    const int M = st->M;
    const size_t n = g.size();
    uint64_t units = uint64_t(1) << (M - 1);
    // one wave: the blocks that fit on the SMs at once (a second, partial wave
    // would leave most SMs idle at the end of every pass)
    int per_sm = 0;
    QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_decoh<T2>, kThreads, 0));
    int grid = int(std::min<uint64_t>((units + kThreads - 1) / kThreads, kMaxParts));
    grid = std::max(1, std::min(grid, std::max(1, per_sm) * num_sms()));
    T2 *amps = static_cast<T2 *>(st->amps);
    for (size_t i = 0; i <= n; ++i) {
        DecohOp op{};
        op.tp = i > 0 ? g[i - 1].t : -1;
        op.t = i < n ? g[i].t : -1;
        op.gamma = gamma;
        op.nparts = grid;
        if (i > 0) {
            op.r_prev = r[i - 1];
            op.idx_prev = int(i - 1);
        }
        if (i < n) {
            op.cmask = g[i].cmask;
            // Rz(delta) . U: row 0 times e^{-i delta/2}, row 1 times e^{+i delta/2}
            const double c = std::cos(0.5 * delta[i]), s = std::sin(0.5 * delta[i]);
            op.rz[0] = c;
            op.rz[1] = s;
            for (int e = 0; e < 4; ++e) {
                const double ur = g[i].U[2 * e], ui = g[i].U[2 * e + 1];
                const double sg = e < 2 ? -s : s;
                op.U[2 * e] = c * ur - sg * ui;
                op.U[2 * e + 1] = c * ui + sg * ur;
            }
        }
        double *prev = d_parts + size_t(((i + 1) & 1)) * 2 * kMaxParts;
        double *cur = d_parts + size_t(i & 1) * 2 * kMaxParts;
        k_decoh<T2><<<grid, kThreads, 0, st->stream>>>(amps, M, op, prev, cur, d_jumps, d_p);
        QS_CHECK_LAUNCH("decoherence launch");
    }
    return QSIM_OK;
}

}  // namespace
}  // namespace qs

extern "C" int qsim_run_decoherence(qsim_state *st, const qsim_gate *gates, size_t n, const double *delta,
                                    const double *r, double gamma, int32_t *jumps, double *p_out) {
    using namespace qs;
    if (!st || !st->amps) { set_error("state is NULL"); return QSIM_EINVAL; }
    if (n > 0 && (!gates || !delta || !r)) { set_error("gates, delta or r is NULL"); return QSIM_EINVAL; }
    if (!(gamma >= 0.0 && gamma <= 1.0)) { set_error("gamma = %g outside [0, 1]", gamma); return QSIM_EINVAL; }
    if (n > size_t(1) << 30) { set_error("too many operations"); return QSIM_EINVAL; }
    std::vector<Gate> g(n);
    for (size_t i = 0; i < n; ++i) {
        if (int rc = make_gate(st->M, gates[i].U, gates[i].target, gates[i].controls, gates[i].ncontrols, &g[i])) {
            char msg[512];
            snprintf(msg, sizeof msg, "gate %zu: %s", i, qsim_last_error());
            set_error("%s", msg);
            return rc;
        }
        if (!std::isfinite(delta[i]) || !std::isfinite(r[i])) {
            set_error("delta or r of operation %zu is not finite", i);
            return QSIM_EINVAL;
        }
    }
    if (n == 0) return QSIM_OK;
    const size_t parts_bytes = 2 * 2 * size_t(kMaxParts) * sizeof(double);
    const size_t out_bytes = n * (sizeof(int) + sizeof(double));
    void *buf = nullptr;
    if (int rc = dmalloc(st->alloc, &buf, parts_bytes + out_bytes, st->stream, "decoherence sums")) return rc;
    double *d_parts = static_cast<double *>(buf);
    double *d_p = d_parts + 4 * size_t(kMaxParts);
    int *d_jumps = reinterpret_cast<int *>(d_p + n);
    int rc = st->prec == QSIM_C64 ? run<float2>(st, g, delta, r, gamma, d_jumps, d_p, d_parts)
                                  : run<double2>(st, g, delta, r, gamma, d_jumps, d_p, d_parts);
    if (rc == QSIM_OK && jumps) {
        cudaError_t e = cudaMemcpyAsync(jumps, d_jumps, n * sizeof(int), cudaMemcpyDeviceToHost, st->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "decoherence jumps");
    }
    if (rc == QSIM_OK && p_out) {
        cudaError_t e = cudaMemcpyAsync(p_out, d_p, n * sizeof(double), cudaMemcpyDeviceToHost, st->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "decoherence probabilities");
    }
    if (rc == QSIM_OK) {
        cudaError_t e = cudaStreamSynchronize(st->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "decoherence run");
    }
    dfree(st->alloc, buf, parts_bytes + out_bytes, st->stream);
    return rc;
}
