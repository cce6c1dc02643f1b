// Device helpers of the specialised tile-pass kernels (compiled at plan
// creation by NVRTC, see jit.cu).  Self-contained: NVRTC sees no host
// headers.  The same arithmetic as cx.cuh and k_tile_reg.cu: Section 2.1's
// pair update with compensated (hi + lo) gate entries, and runs of phase gates
// as a phase polynomial of the index bits in fixed-point turns of 2^-32.

typedef unsigned int qs_u32;
typedef unsigned long long qs_u64;

__device__ __forceinline__ float2 qs_cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// (uh + ul) * a
__device__ __forceinline__ float2 qs_cmulx(float2 uh, float2 ul, float2 a) {
    const float lre = fmaf(ul.x, a.x, -ul.y * a.y);
    const float lim = fmaf(ul.x, a.y, ul.y * a.x);
    return make_float2(fmaf(uh.x, a.x, fmaf(-uh.y, a.y, lre)), fmaf(uh.x, a.y, fmaf(uh.y, a.x, lim)));
}
// (uh + ul) * a + (vh + vl) * b
__device__ __forceinline__ float2 qs_cmad2x(float2 uh, float2 ul, float2 a, float2 vh, float2 vl, float2 b) {
    const float lre = fmaf(ul.x, a.x, fmaf(-ul.y, a.y, fmaf(vl.x, b.x, -vl.y * b.y)));
    const float lim = fmaf(ul.x, a.y, fmaf(ul.y, a.x, fmaf(vl.x, b.y, vl.y * b.x)));
    const float re = fmaf(uh.x, a.x, fmaf(-uh.y, a.y, fmaf(vh.x, b.x, fmaf(-vh.y, b.y, lre))));
    const float im = fmaf(uh.x, a.y, fmaf(uh.y, a.x, fmaf(vh.x, b.y, fmaf(vh.y, b.x, lim))));
    return make_float2(re, im);
}
// real entries (u + ul) a + (w + wl) b per component
__device__ __forceinline__ float2 qs_rmad2x(float u, float ul, float2 a, float w, float wl, float2 b) {
    return make_float2(fmaf(u, a.x, fmaf(w, b.x, fmaf(ul, a.x, wl * b.x))),
                       fmaf(u, a.y, fmaf(w, b.y, fmaf(ul, a.y, wl * b.y))));
}
// e^{2 pi i phi / 2^32}: the top 24 bits through sincospif (exact argument),
// the low 8 bits (< 3.7e-7 rad) as a first-order rotation.
__device__ __forceinline__ float2 qs_expi(qs_u32 phi) {
    const int sp = int(phi);
    const float x = float(sp >> 8) * (1.0f / 8388608.0f);
    float sn, cs;
    sincospif(x, &sn, &cs);
    const float r = float(phi & 255u) * 1.4629180792671596e-09f;
    return make_float2(fmaf(-sn, r, cs), fmaf(cs, r, sn));
}

struct QsPhaseRunHdr {
    qs_u32 M, b, q_offset, pad;
};

// Per-tile constants of a phase-polynomial record (all threads call it; one
// barrier): cl[t] = c_{q_t} + sum over set outside bits k of w[q_t][r_k],
// kt = c0 + sum over set outside bits k <= k2 of (c_{r_k} or w[r_k][r_k2]).
// tq[t] = device position of tile bit t, opos[k] = of outside bit k.
template <int B, int NOUT>
__device__ __forceinline__ void qs_phrun_setup(const unsigned char *__restrict__ rec, qs_u64 tile, const int *tq,
                                               const int *opos, qs_u32 *cl, qs_u32 *ktw) {
    const int M = int(reinterpret_cast<const QsPhaseRunHdr *>(rec)->M);
    const qs_u32 *c = reinterpret_cast<const qs_u32 *>(rec + sizeof(QsPhaseRunHdr)) + 1;
    const qs_u32 *w = c + M;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool set = lane < NOUT && ((tile >> lane) & 1);
    const int r = lane < NOUT ? opos[lane] : 0;
    for (int t = warp; t < B; t += 8) {
        const qs_u32 v = __reduce_add_sync(0xffffffffu, set ? __ldg(w + tq[t] * M + r) : 0u);
        if (lane == 0) cl[t] = v + __ldg(c + tq[t]);
    }
    qs_u32 kv = 0;
    for (int p = threadIdx.x; p < NOUT * NOUT; p += 256) {
        const int k = p / NOUT, k2 = p - k * NOUT;
        if (k2 < k || !((tile >> k) & 1) || !((tile >> k2) & 1)) continue;
        kv += k2 == k ? __ldg(c + opos[k]) : __ldg(w + opos[k] * M + opos[k2]);
    }
    kv = __reduce_add_sync(0xffffffffu, kv);
    if (lane == 0) ktw[warp] = kv;
    __syncthreads();
}

// A gate of an error trajectory (Sections 1.4, 2.0): its error-free matrix,
// the axis n of its error (zero: no error) and its column in the error table.
// Same layout as TrajOp of trajectories.cu.
struct QsTrajOp {
    double U[8];
    double ax[3];
    int gate;
    qs_u32 kind, tl, lmask, pad;
    qs_u64 gmask, gsel;
};

// U . exp(-i e/2 n.sigma) in FP64, split into float hi + lo.
__device__ __forceinline__ void qs_noisy_matrix(const QsTrajOp &op, double e, float2 *u, float2 *ul) {
    double r[8];
    const double nx = op.ax[0], ny = op.ax[1], nz = op.ax[2];
    if (nx == 0.0 && ny == 0.0 && nz == 0.0) {
        for (int k = 0; k < 8; ++k) r[k] = op.U[k];
    } else {
        double sn, cs;
        sincos(0.5 * e, &sn, &cs);
        // E = c I - i s n.sigma = [[c - i s nz, -s ny - i s nx], [s ny - i s nx, c + i s nz]]
        const double E[8] = {cs, -sn * nz, -sn * ny, -sn * nx, sn * ny, -sn * nx, cs, sn * nz};
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double re = 0, im = 0;
                for (int k = 0; k < 2; ++k) {
                    const double ar = op.U[2 * (2 * i + k)], ai = op.U[2 * (2 * i + k) + 1];
                    const double br = E[2 * (2 * k + j)], bi = E[2 * (2 * k + j) + 1];
                    re += ar * br - ai * bi;
                    im += ar * bi + ai * br;
                }
                r[2 * (2 * i + j)] = re;
                r[2 * (2 * i + j) + 1] = im;
            }
    }
    for (int k = 0; k < 4; ++k) {
        const float hr = float(r[2 * k]), hi = float(r[2 * k + 1]);
        u[k] = make_float2(hr, hi);
        ul[k] = make_float2(float(r[2 * k] - double(hr)), float(r[2 * k + 1] - double(hi)));
    }
}
