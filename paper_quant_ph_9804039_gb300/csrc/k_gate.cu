// Single-gate kernels: one launch applies one controlled single-target gate
// to the whole state vector (Section 2.1, Figure 3: the 2x2 operation on
// every pair of states that differ only in the target bit; a controlled gate
// touches only the pairs whose control bits are all one).
//
//   k_gate_hi  target bit >= kLoBits: the pair partners lie in different
//              warps' chunks.  Work items enumerate exactly the touched pairs
//              (target and high control bits inserted), so a gate with c high
//              controls reads and writes 2^(M-c) amplitudes.  Each thread
//              moves 16-byte vectors (two complex64 or one complex128) from
//              both halves of its pairs; a warp covers >= 512 contiguous bytes.
//   k_gate_lo  target bit < kLoBits: a warp owns 512 contiguous bytes of the
//              vector; the partner amplitude sits in the same thread (bit 0 of
//              complex64) or in lane ^ 2^k, fetched with a warp shuffle.
//   k_gate_small  plain one-pair-per-thread form for states too small for
//              the vectorised kernels (M < 8).
//
// Gate kinds (classified on the host): DENSE 2x2; DIAG and PHASE1 multiply
// in place (PHASE1 enumerates only the target-1 states); SWAPX (U = X
// exactly) exchanges the pair without arithmetic, so NOT, CNOT and Toffoli
// are exact permutations.  Control bits below kLoBits are tested per
// amplitude (they would break coalescing if enumerated).
#include "cx.cuh"
#include "qsim_internal.h"

namespace qs {
namespace {

template <typename R>
struct GateK {
    typename CxT<R>::T u00, u01, u10, u11;  // hi parts (the entries, for double)
    typename CxT<R>::T l00, l01, l10, l11;  // lo parts (complex64 only)
    uint64_t lowctl;   // control bits tested per amplitude
    uint64_t setmask;  // bits forced to one after insertion
    int t;
    int nins;
    int ins[3];  // inserted bit positions, ascending
};

__device__ __forceinline__ uint64_t expand(uint64_t p, int nins, const int *ins) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (k < nins) p = insert0(p, ins[k]);
    return p;
}

template <typename T2, typename G>
__device__ __forceinline__ T2 gate_lo_val(uint32_t kind, const G &g, T2 own, T2 partner, bool upper) {
    // upper: this amplitude has target bit 1
    if (kind == K_SWAPX) return partner;
    if (kind == K_DIAG) return upper ? cmulx(g.u11, g.l11, own) : cmulx(g.u00, g.l00, own);
    if (kind == K_PHASE1) return upper ? cmulx(g.u11, g.l11, own) : own;
    return upper ? cmad2x(g.u10, g.l10, partner, g.u11, g.l11, own) : cmad2x(g.u00, g.l00, own, g.u01, g.l01, partner);
}

// ---------------------------------------------------------------- hi
template <uint32_t KIND>
__global__ void __launch_bounds__(256) k_gate_hi_f(float2 *__restrict__ a, uint64_t nitems, GateK<float> g) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x * 2;
    const uint64_t tb = uint64_t(1) << g.t;
    for (uint64_t p = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) * 2; p < nitems; p += stride) {
        const uint64_t i = expand(p, g.nins, g.ins) | g.setmask;  // even: bit 0 of p is 0
        const bool m0 = (i & g.lowctl) == g.lowctl;
        const bool m1 = ((i + 1) & g.lowctl) == g.lowctl;
        if (!m0 && !m1) continue;
        float4 *pi = reinterpret_cast<float4 *>(a + i);
        if (KIND == K_PHASE1) {  // i enumerates the target-1 states
            float4 v = *pi;
            float2 x0 = make_float2(v.x, v.y), x1 = make_float2(v.z, v.w);
            if (m0) x0 = cmulx(g.u11, g.l11, x0);
            if (m1) x1 = cmulx(g.u11, g.l11, x1);
            *pi = make_float4(x0.x, x0.y, x1.x, x1.y);
            continue;
        }
        float4 *pj = reinterpret_cast<float4 *>(a + (i | tb));
        float4 va = *pi, vb = *pj;
        float2 a0 = make_float2(va.x, va.y), a1 = make_float2(va.z, va.w);
        float2 b0 = make_float2(vb.x, vb.y), b1 = make_float2(vb.z, vb.w);
        float2 ra0 = a0, ra1 = a1, rb0 = b0, rb1 = b1;
        if (KIND == K_SWAPX) {
            if (m0) { ra0 = b0; rb0 = a0; }
            if (m1) { ra1 = b1; rb1 = a1; }
        } else if (KIND == K_DIAG) {
            if (m0) { ra0 = cmulx(g.u00, g.l00, a0); rb0 = cmulx(g.u11, g.l11, b0); }
            if (m1) { ra1 = cmulx(g.u00, g.l00, a1); rb1 = cmulx(g.u11, g.l11, b1); }
        } else {
            if (m0) { ra0 = cmad2x(g.u00, g.l00, a0, g.u01, g.l01, b0); rb0 = cmad2x(g.u10, g.l10, a0, g.u11, g.l11, b0); }
            if (m1) { ra1 = cmad2x(g.u00, g.l00, a1, g.u01, g.l01, b1); rb1 = cmad2x(g.u10, g.l10, a1, g.u11, g.l11, b1); }
        }
        *pi = make_float4(ra0.x, ra0.y, ra1.x, ra1.y);
        *pj = make_float4(rb0.x, rb0.y, rb1.x, rb1.y);
    }
}

template <uint32_t KIND>
__global__ void __launch_bounds__(256) k_gate_hi_d(double2 *__restrict__ a, uint64_t nitems, GateK<double> g) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tb = uint64_t(1) << g.t;
    for (uint64_t p = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < nitems; p += stride) {
        const uint64_t i = expand(p, g.nins, g.ins) | g.setmask;
        if ((i & g.lowctl) != g.lowctl) continue;
        if (KIND == K_PHASE1) {
            a[i] = cmul(g.u11, a[i]);
            continue;
        }
        const uint64_t j = i | tb;
        double2 x = a[i], y = a[j];
        if (KIND == K_SWAPX) {
            a[i] = y;
            a[j] = x;
        } else if (KIND == K_DIAG) {
            a[i] = cmul(g.u00, x);
            a[j] = cmul(g.u11, y);
        } else {
            a[i] = cmad2(g.u00, x, g.u01, y);
            a[j] = cmad2(g.u10, x, g.u11, y);
        }
    }
}

// ---------------------------------------------------------------- lo
// nitems = thread items (each 16 bytes of the vector); a multiple of 32, so a
// warp always runs the loop body together (the shuffles need all lanes).
template <uint32_t KIND>
__global__ void __launch_bounds__(256) k_gate_lo_f(float2 *__restrict__ a, uint64_t nitems, GateK<float> g) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t q = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < nitems; q += stride) {
        const uint64_t i = expand(q * 2, g.nins, g.ins) | g.setmask;
        float4 *pi = reinterpret_cast<float4 *>(a + i);
        float4 v = *pi;
        float2 x0 = make_float2(v.x, v.y), x1 = make_float2(v.z, v.w);
        const bool m0 = (i & g.lowctl) == g.lowctl;
        const bool m1 = ((i + 1) & g.lowctl) == g.lowctl;
        float2 r0 = x0, r1 = x1;
        if (g.t == 0) {
            if (KIND == K_SWAPX) {
                if (m0) { r0 = x1; r1 = x0; }
            } else if (KIND == K_DIAG) {
                if (m0) { r0 = cmulx(g.u00, g.l00, x0); r1 = cmulx(g.u11, g.l11, x1); }
            } else if (KIND == K_PHASE1) {
                if (m0) r1 = cmulx(g.u11, g.l11, x1);
            } else {
                if (m0) { r0 = cmad2x(g.u00, g.l00, x0, g.u01, g.l01, x1); r1 = cmad2x(g.u10, g.l10, x0, g.u11, g.l11, x1); }
            }
        } else {
            const bool upper = (i >> g.t) & 1;
            float2 w0 = x0, w1 = x1;
            if (KIND == K_DENSE || KIND == K_SWAPX) {
                const int lm = 1 << (g.t - 1);
                w0.x = __shfl_xor_sync(0xffffffffu, x0.x, lm);
                w0.y = __shfl_xor_sync(0xffffffffu, x0.y, lm);
                w1.x = __shfl_xor_sync(0xffffffffu, x1.x, lm);
                w1.y = __shfl_xor_sync(0xffffffffu, x1.y, lm);
            }
            if (m0) r0 = gate_lo_val(KIND, g, x0, w0, upper);
            if (m1) r1 = gate_lo_val(KIND, g, x1, w1, upper);
        }
        *pi = make_float4(r0.x, r0.y, r1.x, r1.y);
    }
}

template <uint32_t KIND>
__global__ void __launch_bounds__(256) k_gate_lo_d(double2 *__restrict__ a, uint64_t nitems, GateK<double> g) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t q = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < nitems; q += stride) {
        const uint64_t i = expand(q, g.nins, g.ins) | g.setmask;
        double2 x = a[i];
        const bool m = (i & g.lowctl) == g.lowctl;
        const bool upper = (i >> g.t) & 1;
        double2 w = x;
        if (KIND == K_DENSE || KIND == K_SWAPX) {
            const int lm = 1 << g.t;
            w.x = __shfl_xor_sync(0xffffffffu, x.x, lm);
            w.y = __shfl_xor_sync(0xffffffffu, x.y, lm);
        }
        if (m) a[i] = gate_lo_val(KIND, g, x, w, upper);
    }
}

// ---------------------------------------------------------------- small
template <typename R>
__global__ void k_gate_small(typename CxT<R>::T *__restrict__ a, int M, uint32_t kind, GateK<R> g,
                             uint64_t cmask) {
    using T2 = typename CxT<R>::T;
    const uint64_t npairs = uint64_t(1) << (M - 1);
    const uint64_t tb = uint64_t(1) << g.t;
    for (uint64_t p = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < npairs;
         p += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t i = insert0(p, g.t);
        if ((i & cmask) != cmask) continue;
        const uint64_t j = i | tb;
        T2 x = a[i], y = a[j];
        if (kind == K_SWAPX) {
            a[i] = y;
            a[j] = x;
        } else if (kind == K_DIAG || kind == K_PHASE1) {
            a[i] = cmulx(g.u00, g.l00, x);
            a[j] = cmulx(g.u11, g.l11, y);
        } else {
            a[i] = cmad2x(g.u00, g.l00, x, g.u01, g.l01, y);
            a[j] = cmad2x(g.u10, g.l10, x, g.u11, g.l11, y);
        }
    }
}

template <typename R>
GateK<R> make_k(const Gate &g) {
    GateK<R> k{};
    typename CxT<R>::T *hi[4] = {&k.u00, &k.u01, &k.u10, &k.u11};
    typename CxT<R>::T *lo[4] = {&k.l00, &k.l01, &k.l10, &k.l11};
    for (int e = 0; e < 4; ++e) {
        if constexpr (sizeof(R) == 4) {
            float hr, lr, hi_, li;
            split_f(g.U[2 * e], hr, lr);
            split_f(g.U[2 * e + 1], hi_, li);
            *hi[e] = mk(hr, hi_);
            *lo[e] = mk(lr, li);
        } else {
            *hi[e] = mk(R(g.U[2 * e]), R(g.U[2 * e + 1]));
            *lo[e] = mk(R(0), R(0));
        }
    }
    k.t = g.t;
    return k;
}

inline unsigned grid_for(uint64_t items, int per_block) {
    uint64_t blocks = (items + per_block - 1) / per_block;
    uint64_t cap = uint64_t(num_sms()) * 32;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return unsigned(blocks);
}

// Split controls into inserted (>= lob) and per-amplitude (< lob) ones.
template <typename R>
void place_bits(const Gate &g, int lob, bool insert_target, GateK<R> &k) {
    int pos[3];
    int n = 0;
    if (insert_target) pos[n++] = g.t;
    for (int c = 0; c < g.nc; ++c) {
        if (g.c[c] >= lob) {
            pos[n++] = g.c[c];
            k.setmask |= uint64_t(1) << g.c[c];
        } else {
            k.lowctl |= uint64_t(1) << g.c[c];
        }
    }
    for (int x = 0; x < n; ++x)
        for (int y = x + 1; y < n; ++y)
            if (pos[y] < pos[x]) { int tmp = pos[x]; pos[x] = pos[y]; pos[y] = tmp; }
    k.nins = n;
    for (int x = 0; x < n; ++x) k.ins[x] = pos[x];
}

}  // namespace

#define QS_DISPATCH_KIND(KERN, kind, grid, a, items, k, s)                       \
    switch (kind) {                                                              \
        case K_SWAPX: KERN<K_SWAPX><<<grid, 256, 0, s>>>(a, items, k); break;   \
        case K_DIAG: KERN<K_DIAG><<<grid, 256, 0, s>>>(a, items, k); break;     \
        case K_PHASE1: KERN<K_PHASE1><<<grid, 256, 0, s>>>(a, items, k); break; \
        default: KERN<K_DENSE><<<grid, 256, 0, s>>>(a, items, k); break;        \
    }

int launch_gate(void *amps, int M, qsim_prec prec, const Gate &g, cudaStream_t s) {
    if (prec == QSIM_C64) {
        float2 *a = static_cast<float2 *>(amps);
        const int lob = 6;
        if (M < 8) {
            GateK<float> k = make_k<float>(g);
            k_gate_small<float><<<grid_for(uint64_t(1) << (M - 1), 256), 256, 0, s>>>(a, M, g.kind, k, g.cmask);
        } else if (g.t >= lob) {
            GateK<float> k = make_k<float>(g);
            place_bits(g, lob, true, k);
            if (g.kind == K_PHASE1) k.setmask |= uint64_t(1) << g.t;
            const uint64_t items = uint64_t(1) << (M - k.nins);
            QS_DISPATCH_KIND(k_gate_hi_f, g.kind, grid_for(items / 2, 256), a, items, k, s);
        } else {
            GateK<float> k = make_k<float>(g);
            place_bits(g, lob, false, k);
            const uint64_t items = uint64_t(1) << (M - k.nins - 1);  // 16-byte items
            QS_DISPATCH_KIND(k_gate_lo_f, g.kind, grid_for(items, 256), a, items, k, s);
        }
    } else {
        double2 *a = static_cast<double2 *>(amps);
        const int lob = 5;
        if (M < 8) {
            GateK<double> k = make_k<double>(g);
            k_gate_small<double><<<grid_for(uint64_t(1) << (M - 1), 256), 256, 0, s>>>(a, M, g.kind, k, g.cmask);
        } else if (g.t >= lob) {
            GateK<double> k = make_k<double>(g);
            place_bits(g, lob, true, k);
            if (g.kind == K_PHASE1) k.setmask |= uint64_t(1) << g.t;
            const uint64_t items = uint64_t(1) << (M - k.nins);
            QS_DISPATCH_KIND(k_gate_hi_d, g.kind, grid_for(items, 256), a, items, k, s);
        } else {
            GateK<double> k = make_k<double>(g);
            place_bits(g, lob, false, k);
            const uint64_t items = uint64_t(1) << (M - k.nins);
            QS_DISPATCH_KIND(k_gate_lo_d, g.kind, grid_for(items, 256), a, items, k, s);
        }
    }
    QS_CHECK_LAUNCH("single-gate kernel launch");
    return QSIM_OK;
}

}  // namespace qs
