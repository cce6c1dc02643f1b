/*
 * qsim_oracle.c -- plain CPU complex128 reference of the error-injecting
 * state-vector simulator (Obenland & Despain, "A Parallel Quantum Computer
 * Simulator").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header or constant with the CUDA path and includes none of its files.
 *
 * What it computes (all in double precision complex):
 *   - Section 1.2: a register of M qubits is a vector of 2^M complex
 *     amplitudes; the index of an amplitude is the bit value of its basis
 *     state; the probability of a state is |amplitude|^2.
 *   - Section 1.3: a gate is a 2^M x 2^M matrix times the vector.
 *   - Section 2.1 (Figure 3): because a gate acts on few bits, the big matrix
 *     is a 2x2 block replicated; the simulator applies the 2x2 operation to
 *     every pair of states whose indices differ only in the target bit.  A
 *     controlled gate (Section 1.3, Table 1 / Figure 2; Section 2.0's one-,
 *     two- and three-bit controlled-NOTs) applies it only to the pairs whose
 *     control bits are all one.
 *   - Sections 1.4 / 2.0: operational errors are deviations of the rotation
 *     angle; for a gate with rotation axis n the erroneous gate is
 *     U . exp(-i eps/2 n.sigma).
 *   - Fidelity of a noisy run against the error-free run:
 *     F = |sum_i conj(ideal_i) noisy_i|^2, norm = sum_i |noisy_i|^2.
 *
 * Pins (tests marked "not gpu"): brute-force 2^M x 2^M Kronecker products,
 * the Figure 1 and Table 1 / Figure 2 examples, norm preservation, the
 * uniform superposition, circuit-then-inverse, the QFT closed form, the
 * single-error closed form F = cos^2(eps/2), and mutants of this file.
 *
 * Work over the 2^M indices may be split across host threads by contiguous
 * index ranges; a pair is updated only by the thread that owns its lower
 * index, so no two threads touch the same amplitude.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ gates */

/* One gate: (a_i, a_j) <- (U00 a_i + U01 a_j, U10 a_i + U11 a_j) for every
 * index i whose target bit is 0 and whose control bits are all 1, with
 * j = i | 2^target (Section 2.1, Figure 3).  U is row-major, re/im interleaved. */
static void gate_range(cplx *psi, const double *U, int target, uint64_t ctl_mask,
                       uint64_t lo, uint64_t hi)
{
    const cplx u00 = U[0] + I * U[1], u01 = U[2] + I * U[3];
    const cplx u10 = U[4] + I * U[5], u11 = U[6] + I * U[7];
    const uint64_t tbit = (uint64_t)1 << target;
    for (uint64_t i = lo; i < hi; ++i) {
        if (i & tbit) continue;
        if ((i & ctl_mask) != ctl_mask) continue;
        uint64_t j = i | tbit;
        cplx a = psi[i], b = psi[j];
        psi[i] = u00 * a + u01 * b;
        psi[j] = u10 * a + u11 * b;
    }
}

struct gate_job {
    cplx *psi; const double *U; int target; uint64_t ctl_mask; uint64_t lo, hi;
};

static void *gate_thread(void *p)
{
    struct gate_job *j = (struct gate_job *)p;
    gate_range(j->psi, j->U, j->target, j->ctl_mask, j->lo, j->hi);
    return NULL;
}

static int check_gate(int M, int target, const int *ctl, int nctl)
{
    if (M < 1 || M > 40) return -1;
    if (target < 0 || target >= M) return -1;
    if (nctl < 0 || nctl > 2) return -1;
    for (int c = 0; c < nctl; ++c) {
        if (ctl[c] < 0 || ctl[c] >= M || ctl[c] == target) return -1;
        for (int d = 0; d < c; ++d) if (ctl[d] == ctl[c]) return -1;
    }
    return 0;
}

int orc_apply_gate(double *psi_ri, int M, const double *U, int target,
                   const int *ctl, int nctl, int nthreads)
{
    if (check_gate(M, target, ctl, nctl)) return -1;
    cplx *psi = (cplx *)psi_ri;
    uint64_t ctl_mask = 0;
    for (int c = 0; c < nctl; ++c) ctl_mask |= (uint64_t)1 << ctl[c];
    const uint64_t N = (uint64_t)1 << M;
    if (nthreads <= 1 || N < 4096) {
        gate_range(psi, U, target, ctl_mask, 0, N);
        return 0;
    }
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    struct gate_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].psi = psi; jobs[t].U = U; jobs[t].target = target; jobs[t].ctl_mask = ctl_mask;
        jobs[t].lo = N * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = N * (uint64_t)(t + 1) / (uint64_t)nthreads;
        pthread_create(&th[t], NULL, gate_thread, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* Gates applied one after the other, in the order given. */
int orc_apply_gates(double *psi_ri, int M, int64_t n, const double *U /* [n][8] */,
                    const int *target, const int *nctl, const int *ctl /* [n][2] */,
                    int nthreads)
{
    for (int64_t g = 0; g < n; ++g) {
        int rc = orc_apply_gate(psi_ri, M, U + 8 * g, target[g], ctl + 2 * g, nctl[g], nthreads);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------- reductions */

/* norm = sum_i |psi_i|^2 (Section 1.2: the probabilities sum to one). */
double orc_norm(const double *psi_ri, int64_t N)
{
    const cplx *psi = (const cplx *)psi_ri;
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    return s;
}

/* out = sum_i conj(a_i) b_i */
void orc_overlap(const double *a_ri, const double *b_ri, int64_t N, double *out)
{
    const cplx *a = (const cplx *)a_ri, *b = (const cplx *)b_ri;
    cplx s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += conj(a[i]) * b[i];
    out[0] = creal(s);
    out[1] = cimag(s);
}

/* F = |<ideal|noisy>|^2 (raw, not renormalised) and the norm of noisy. */
void orc_fidelity(const double *ideal_ri, const double *noisy_ri, int64_t N,
                  double *F, double *norm_noisy)
{
    double ov[2];
    orc_overlap(ideal_ri, noisy_ri, N, ov);
    *F = ov[0] * ov[0] + ov[1] * ov[1];
    *norm_noisy = orc_norm(noisy_ri, N);
}

/* p_i = |psi_i|^2 (Section 1.2, Figure 1). */
void orc_probabilities(const double *psi_ri, int64_t N, double *p)
{
    const cplx *psi = (const cplx *)psi_ri;
    for (int64_t i = 0; i < N; ++i) p[i] = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
}

/* ---------------------------------------------------------- error gates */

/* out = U . exp(-i eps/2 (nx X + ny Y + nz Z)): the gate with its rotation
 * angle deviated by eps about the axis n (Sections 1.4, 2.0).  n = 0 leaves
 * the gate unchanged. */
void orc_error_gate(const double *U, const double *axis, double eps, double *out)
{
    const double nx = axis[0], ny = axis[1], nz = axis[2];
    if (nx == 0.0 && ny == 0.0 && nz == 0.0) {
        memcpy(out, U, 8 * sizeof(double));
        return;
    }
    const cplx u00 = U[0] + I * U[1], u01 = U[2] + I * U[3];
    const cplx u10 = U[4] + I * U[5], u11 = U[6] + I * U[7];
    const double c = cos(0.5 * eps), s = sin(0.5 * eps);
    /* E = c I - i s (n.sigma), n.sigma = [[nz, nx - i ny], [nx + i ny, -nz]] */
    const cplx e00 = c - I * s * nz;
    const cplx e01 = -I * s * (nx - I * ny);
    const cplx e10 = -I * s * (nx + I * ny);
    const cplx e11 = c + I * s * nz;
    const cplx r00 = u00 * e00 + u01 * e10, r01 = u00 * e01 + u01 * e11;
    const cplx r10 = u10 * e00 + u11 * e10, r11 = u10 * e01 + u11 * e11;
    out[0] = creal(r00); out[1] = cimag(r00); out[2] = creal(r01); out[3] = cimag(r01);
    out[4] = creal(r10); out[5] = cimag(r10); out[6] = creal(r11); out[7] = cimag(r11);
}

/* ----------------------------------------------------------- trajectories */

struct traj_job {
    int M; int64_t n; const double *U; const int *target; const int *nctl; const int *ctl;
    const double *axis; const double *eps; const double *ideal; double *F;
    int t0, t1;
};

static void *traj_thread(void *p)
{
    struct traj_job *j = (struct traj_job *)p;
    const uint64_t N = (uint64_t)1 << j->M;
    double *psi = (double *)malloc(sizeof(double) * 2 * N);
    double Ue[8];
    for (int t = j->t0; t < j->t1; ++t) {
        memset(psi, 0, sizeof(double) * 2 * N);
        psi[0] = 1.0;                                   /* |0...0> */
        for (int64_t g = 0; g < j->n; ++g) {
            orc_error_gate(j->U + 8 * g, j->axis + 3 * g, j->eps[(int64_t)t * j->n + g], Ue);
            orc_apply_gate(psi, j->M, Ue, j->target[g], j->ctl + 2 * g, j->nctl[g], 1);
        }
        double nrm;
        orc_fidelity(j->ideal, psi, (int64_t)N, &j->F[t], &nrm);
    }
    free(psi);
    return NULL;
}

/* T error trajectories of one circuit, each started from |0...0>, each gate g
 * of trajectory t deviated by eps[t][g] about axis[g].  F[t] is the fidelity
 * against the error-free run; mean and unbiased variance of F over t. */
int orc_trajectories(int M, int64_t n, const double *U, const int *target, const int *nctl,
                     const int *ctl, const double *axis, const double *eps, int T,
                     double *F, double *mean, double *var, int nthreads)
{
    if (M < 1 || M > 30 || T < 1) return -1;
    for (int64_t g = 0; g < n; ++g)
        if (check_gate(M, target[g], ctl + 2 * g, nctl[g])) return -1;
    const uint64_t N = (uint64_t)1 << M;
    double *ideal = (double *)calloc(2 * N, sizeof(double));
    ideal[0] = 1.0;
    orc_apply_gates(ideal, M, n, U, target, nctl, ctl, 1);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > T) nthreads = T;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    struct traj_job jobs[256];
    for (int k = 0; k < nthreads; ++k) {
        struct traj_job jj = {M, n, U, target, nctl, ctl, axis, eps, ideal, F,
                              (int)((int64_t)T * k / nthreads), (int)((int64_t)T * (k + 1) / nthreads)};
        jobs[k] = jj;
        pthread_create(&th[k], NULL, traj_thread, &jobs[k]);
    }
    for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
    double s = 0.0;
    for (int t = 0; t < T; ++t) s += F[t];
    *mean = s / T;
    double v = 0.0;
    for (int t = 0; t < T; ++t) v += (F[t] - *mean) * (F[t] - *mean);
    *var = (T > 1) ? v / (T - 1) : 0.0;
    free(ideal);
    return 0;
}

/* ------------------------------------------------------------ decoherence */

/* Weights of the qubit's 1 states and of all states: P1 = sum over i with
 * bit t set of |psi_i|^2, N = sum_i |psi_i|^2. */
static void weights(const cplx *psi, int M, int t, double *P1, double *N)
{
    const uint64_t n = (uint64_t)1 << M, tb = (uint64_t)1 << t;
    double p1 = 0.0, all = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        const double w = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        all += w;
        if (i & tb) p1 += w;
    }
    *P1 = p1;
    *N = all;
}

/* Decoherence after every operation (Section 3.4: two more transformations
 * after each operation and a sum over the whole state; EQ 3, EQ 8).  The
 * paper does not give the transformations; the reading taken here: after
 * gate g on target t,
 *   1. dephasing: Rz(delta_g) = diag(e^{-i delta/2}, e^{+i delta/2}) on t;
 *   2. amplitude damping as a quantum jump on t: with P1 and N the weights
 *      above, p = gamma P1 / N is the jump probability; if r_g < p the jump
 *      operator [[0, sqrt(gamma)], [0, 0]] is applied, else the no-jump
 *      operator diag(1, sqrt(1 - gamma)), each scaled so that the norm stays
 *      N: by sqrt(N / (gamma P1)), or sqrt(N / (N - gamma P1)).
 * delta and r come from the caller (seeded); jumps[g] and p_out[g] (may be
 * NULL) receive the decision and p. */
int orc_decoherence(double *psi_ri, int M, int64_t n, const double *U, const int *target, const int *nctl,
                    const int *ctl, const double *delta, const double *r, double gamma, int *jumps,
                    double *p_out, int nthreads)
{
    if (gamma < 0.0 || gamma > 1.0) return -1;
    cplx *psi = (cplx *)psi_ri;
    for (int64_t g = 0; g < n; ++g) {
        const int t = target[g];
        if (orc_apply_gate(psi_ri, M, U + 8 * g, t, ctl + 2 * g, nctl[g], nthreads)) return -1;
        const double h = 0.5 * delta[g];
        const double Rz[8] = {cos(h), -sin(h), 0, 0, 0, 0, cos(h), sin(h)};
        orc_apply_gate(psi_ri, M, Rz, t, NULL, 0, nthreads);
        double P1, N;
        weights(psi, M, t, &P1, &N);
        const double p = N > 0.0 ? gamma * P1 / N : 0.0;
        const int jump = r[g] < p;
        double K[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (jump) {
            K[2] = sqrt(gamma) * sqrt(N / (gamma * P1));
        } else {
            const double s = sqrt(N / (N - gamma * P1));
            K[0] = s;
            K[6] = sqrt(1.0 - gamma) * s;
        }
        orc_apply_gate(psi_ri, M, K, t, NULL, 0, nthreads);
        if (jumps) jumps[g] = jump;
        if (p_out) p_out[g] = p;
    }
    return 0;
}

/* ----------------------------------------------------------------- qutrits */

/* The three-state model (Section 2.0, Section 3.0-3.1): M three-level
 * particles, 3^M complex amplitudes, the index written in base 3 with digit q
 * the level of particle q (digit 0 least significant).  A transformation on
 * one particle is a 3x3 matrix U applied to every triple of states that
 * differ only in that particle's level: (a_i, a_{i + 3^t}, a_{i + 2 3^t}) for
 * every i whose digit t is 0.  A control (c, v) restricts it to the triples
 * whose digit c equals v.  U is row-major, re/im interleaved (18 doubles). */
int orc_qutrit_apply(double *psi_ri, int M, int64_t n, const double *U /* [n][18] */, const int *target,
                     const int *nctl, const int *ctl /* [n][2] */, const int *lvl /* [n][2] */)
{
    if (M < 1 || M > 24) return -1;
    cplx *psi = (cplx *)psi_ri;
    uint64_t pw[26];
    pw[0] = 1;
    for (int q = 1; q <= M; ++q) pw[q] = pw[q - 1] * 3;
    for (int64_t g = 0; g < n; ++g) {
        const int t = target[g];
        if (t < 0 || t >= M || nctl[g] < 0 || nctl[g] > 2) return -1;
        for (int k = 0; k < nctl[g]; ++k) {
            const int c = ctl[2 * g + k], v = lvl[2 * g + k];
            if (c < 0 || c >= M || c == t || v < 0 || v > 2) return -1;
            if (k == 1 && c == ctl[2 * g]) return -1;
        }
        const double *u = U + 18 * g;
        cplx m[9];
        for (int e = 0; e < 9; ++e) m[e] = u[2 * e] + I * u[2 * e + 1];
        for (uint64_t i = 0; i < pw[M]; ++i) {
            if ((i / pw[t]) % 3 != 0) continue;
            int on = 1;
            for (int k = 0; k < nctl[g]; ++k)
                if ((int)((i / pw[ctl[2 * g + k]]) % 3) != lvl[2 * g + k]) on = 0;
            if (!on) continue;
            const cplx a = psi[i], b = psi[i + pw[t]], c = psi[i + 2 * pw[t]];
            psi[i] = m[0] * a + m[1] * b + m[2] * c;
            psi[i + pw[t]] = m[3] * a + m[4] * b + m[5] * c;
            psi[i + 2 * pw[t]] = m[6] * a + m[7] * b + m[8] * c;
        }
    }
    return 0;
}
