// C ABI: states, single gates, reductions, errors.  Plans live in plan.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "qsim_internal.h"

namespace qs {

namespace {
thread_local char g_err[512] = "";
}

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what) {
    set_error("CUDA error %d (%s) in %s", int(e), cudaGetErrorString(e), what);
    cudaGetLastError();  // a non-sticky error is reported once, not again by the next launch check
    return e == cudaErrorMemoryAllocation ? QSIM_ENOMEM : QSIM_ECUDA;
}

int num_sms() {
    static int cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        cache[dev] = v;
    }
    return cache[dev];
}

int make_gate(int M, const double *U, int target, const int *controls, int ncontrols, Gate *out) {
    if (!U) { set_error("gate matrix is NULL"); return QSIM_EINVAL; }
    if (target < 0 || target >= M) { set_error("target %d outside [0, %d)", target, M); return QSIM_EINVAL; }
    if (ncontrols < 0 || ncontrols > 2) { set_error("ncontrols %d outside 0..2", ncontrols); return QSIM_EINVAL; }
    if (ncontrols > 0 && !controls) { set_error("controls is NULL"); return QSIM_EINVAL; }
    Gate g{};
    g.t = target;
    g.nc = ncontrols;
    for (int c = 0; c < ncontrols; ++c) {
        const int q = controls[c];
        if (q < 0 || q >= M) { set_error("control %d outside [0, %d)", q, M); return QSIM_EINVAL; }
        if (q == target) { set_error("control %d equals the target", q); return QSIM_EINVAL; }
        if (g.cmask & (uint64_t(1) << q)) { set_error("control %d repeated", q); return QSIM_EINVAL; }
        g.c[c] = q;
        g.cmask |= uint64_t(1) << q;
    }
    for (int k = 0; k < 8; ++k) {
        if (!std::isfinite(U[k])) { set_error("gate matrix entry %d is not finite", k); return QSIM_EINVAL; }
        g.U[k] = U[k];
    }
    const bool off0 = U[2] == 0.0 && U[3] == 0.0 && U[4] == 0.0 && U[5] == 0.0;
    const bool diag0 = U[0] == 0.0 && U[1] == 0.0 && U[6] == 0.0 && U[7] == 0.0;
    if (off0)
        g.kind = (U[0] == 1.0 && U[1] == 0.0) ? K_PHASE1 : K_DIAG;
    else if (diag0 && U[2] == 1.0 && U[3] == 0.0 && U[4] == 1.0 && U[5] == 0.0)
        g.kind = K_SWAPX;
    else
        g.kind = K_DENSE;
    *out = g;
    return QSIM_OK;
}

double gate_bytes(const Gate &g, int M, size_t ab) {
    double touched = std::ldexp(1.0, M - g.nc);
    if (g.kind == K_PHASE1) touched *= 0.5;
    return 2.0 * touched * double(ab);
}

static int check_state(const qsim_state *st) {
    if (!st) { set_error("state is NULL"); return QSIM_EINVAL; }
    return QSIM_OK;
}

}  // namespace qs

using namespace qs;

static int state_common(int M, qsim_prec prec, qsim_state **out) {
    if (!out) { set_error("out is NULL"); return QSIM_EINVAL; }
    if (M < 1 || M > QSIM_MAX_QUBITS) { set_error("M = %d outside [1, %d]", M, QSIM_MAX_QUBITS); return QSIM_EINVAL; }
    if (prec != QSIM_C64 && prec != QSIM_C128) { set_error("unknown precision %d", int(prec)); return QSIM_EINVAL; }
    return QSIM_OK;
}

static int state_scratch(qsim_state *st) {
    st->scratch_blocks = kReduceSlots;
    if (int rc = dmalloc(st->alloc, reinterpret_cast<void **>(&st->scratch), state_scratch_bytes(kReduceSlots),
                         nullptr, "reduction scratch"))
        return rc;
    QS_CUDA(cudaEventCreateWithFlags(&st->ev, cudaEventDisableTiming));
    return QSIM_OK;
}

extern "C" {

const char *qsim_last_error(void) { return g_err; }

const char *qsim_version(void) { return "qsim-gb300 0.1 (sm_103a)"; }

int qsim_alloc(int M, qsim_prec prec, qsim_state **out) {
    int rc = state_common(M, prec, out);
    if (rc) return rc;
    qsim_state *st = new qsim_state();
    st->M = M;
    st->prec = prec;
    st->owned = true;
    st->stream = nullptr;
    st->alloc = current_allocator();
    if (dmalloc(st->alloc, &st->amps, (size_t(1) << M) * amp_bytes(prec), nullptr, "state amplitudes")) {
        delete st;
        set_error("cannot allocate %zu bytes for a %d-qubit state", (size_t(1) << M) * amp_bytes(prec), M);
        return QSIM_ENOMEM;
    }
    if ((rc = state_scratch(st)) != QSIM_OK || (rc = launch_zero_state(st->amps, M, prec, nullptr)) != QSIM_OK) {
        qsim_free(st);
        return rc;
    }
    *out = st;
    return QSIM_OK;
}

int qsim_wrap(void *device_amps, int M, qsim_prec prec, qsim_state **out) {
    int rc = state_common(M, prec, out);
    if (rc) return rc;
    if (!device_amps || (reinterpret_cast<uintptr_t>(device_amps) & 15)) {
        set_error("device amplitudes must be non-NULL and 16-byte aligned");
        return QSIM_EINVAL;
    }
    qsim_state *st = new qsim_state();
    st->M = M;
    st->prec = prec;
    st->owned = false;
    st->amps = device_amps;
    st->stream = nullptr;
    st->alloc = current_allocator();
    if ((rc = state_scratch(st)) != QSIM_OK) {
        qsim_free(st);
        return rc;
    }
    *out = st;
    return QSIM_OK;
}

void qsim_free(qsim_state *st) {
    if (!st) return;
    cudaStreamSynchronize(st->stream);
    if (st->owned) dfree(st->alloc, st->amps, (size_t(1) << st->M) * amp_bytes(st->prec), nullptr);
    dfree(st->alloc, st->scratch, state_scratch_bytes(st->scratch_blocks), nullptr);
    if (st->ev) cudaEventDestroy(st->ev);
    delete st;
}

int qsim_set_stream(qsim_state *st, void *cuda_stream) {
    if (int rc = check_state(st)) return rc;
    st->stream = static_cast<cudaStream_t>(cuda_stream);
    return QSIM_OK;
}

int qsim_state_info(const qsim_state *st, int *M, int *prec, void **device_amps) {
    if (int rc = check_state(st)) return rc;
    if (M) *M = st->M;
    if (prec) *prec = int(st->prec);
    if (device_amps) *device_amps = st->amps;
    return QSIM_OK;
}

int qsim_reset(qsim_state *st) {
    if (int rc = check_state(st)) return rc;
    return launch_zero_state(st->amps, st->M, st->prec, st->stream);
}

static int copy_in(void *dst, const void *src, size_t bytes, bool on_device, cudaStream_t s) {
    QS_CUDA(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return QSIM_OK;
}

int qsim_set_state(qsim_state *st, const void *amps, int on_device) {
    if (int rc = check_state(st)) return rc;
    if (!amps) { set_error("amps is NULL"); return QSIM_EINVAL; }
    const size_t bytes = (size_t(1) << st->M) * amp_bytes(st->prec);
    if (int rc = copy_in(st->amps, amps, bytes, on_device != 0, st->stream)) return rc;
    if (!on_device) QS_CUDA(cudaStreamSynchronize(st->stream));
    return QSIM_OK;
}

int qsim_set_state_async(qsim_state *st, const void *amps, int on_device) {
    if (int rc = check_state(st)) return rc;
    if (!amps) { set_error("amps is NULL"); return QSIM_EINVAL; }
    const size_t bytes = (size_t(1) << st->M) * amp_bytes(st->prec);
    return copy_in(st->amps, amps, bytes, on_device != 0, st->stream);
}

int qsim_get_state(const qsim_state *st, void *amps, int on_device) {
    if (int rc = check_state(st)) return rc;
    if (!amps) { set_error("amps is NULL"); return QSIM_EINVAL; }
    const size_t bytes = (size_t(1) << st->M) * amp_bytes(st->prec);
    QS_CUDA(cudaMemcpyAsync(amps, st->amps, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            st->stream));
    if (!on_device) QS_CUDA(cudaStreamSynchronize(st->stream));
    return QSIM_OK;
}

int qsim_copy_state(qsim_state *dst, const qsim_state *src) {
    if (int rc = check_state(dst)) return rc;
    if (int rc = check_state(src)) return rc;
    if (dst->M != src->M || dst->prec != src->prec) { set_error("states differ in M or precision"); return QSIM_EINVAL; }
    if (dst == src) return QSIM_OK;
    if (src->stream != dst->stream) {
        QS_CUDA(cudaEventRecord(src->ev, src->stream));
        QS_CUDA(cudaStreamWaitEvent(dst->stream, src->ev, 0));
    }
    QS_CUDA(cudaMemcpyAsync(dst->amps, src->amps, (size_t(1) << dst->M) * amp_bytes(dst->prec),
                            cudaMemcpyDeviceToDevice, dst->stream));
    return QSIM_OK;
}

int qsim_apply_gate(qsim_state *st, const double U[8], int target, const int *controls, int ncontrols) {
    if (int rc = check_state(st)) return rc;
    Gate g;
    if (int rc = make_gate(st->M, U, target, controls, ncontrols, &g)) return rc;
    return launch_gate(st->amps, st->M, st->prec, g, st->stream);
}

int qsim_overlap(const qsim_state *ideal, const qsim_state *noisy, double out[3]) {
    if (!out) { set_error("out is NULL"); return QSIM_EINVAL; }
    if (int rc = check_state(ideal)) return rc;
    if (int rc = check_state(noisy)) return rc;
    if (ideal->M != noisy->M || ideal->prec != noisy->prec) {
        set_error("states differ in M or precision");
        return QSIM_EINVAL;
    }
    if (ideal->stream != noisy->stream) {
        QS_CUDA(cudaEventRecord(ideal->ev, ideal->stream));
        QS_CUDA(cudaStreamWaitEvent(noisy->stream, ideal->ev, 0));
    }
    if (int rc = launch_reduce(ideal->amps, noisy->amps, noisy->M, noisy->prec, noisy->scratch,
                               noisy->scratch_blocks, noisy->stream))
        return rc;
    QS_CUDA(cudaMemcpyAsync(out, noisy->scratch + 3 * size_t(noisy->scratch_blocks), 3 * sizeof(double),
                            cudaMemcpyDeviceToHost, noisy->stream));
    QS_CUDA(cudaStreamSynchronize(noisy->stream));
    return QSIM_OK;
}

int qsim_fidelity(const qsim_state *ideal, const qsim_state *noisy, double *F, double *norm_noisy) {
    if (int rc = check_state(ideal)) return rc;
    if (int rc = check_state(noisy)) return rc;
    if (ideal->M != noisy->M || ideal->prec != noisy->prec) {
        set_error("states differ in M or precision");
        return QSIM_EINVAL;
    }
    if (ideal->stream != noisy->stream) {
        QS_CUDA(cudaEventRecord(ideal->ev, ideal->stream));
        QS_CUDA(cudaStreamWaitEvent(noisy->stream, ideal->ev, 0));
    }
    if (int rc = launch_reduce(ideal->amps, noisy->amps, noisy->M, noisy->prec, noisy->scratch,
                               noisy->scratch_blocks, noisy->stream))
        return rc;
    double r[3];
    QS_CUDA(cudaMemcpyAsync(r, noisy->scratch + 3 * size_t(noisy->scratch_blocks), sizeof(r),
                            cudaMemcpyDeviceToHost, noisy->stream));
    QS_CUDA(cudaStreamSynchronize(noisy->stream));
    if (F) *F = r[1] * r[1] + r[2] * r[2];
    if (norm_noisy) *norm_noisy = r[0];
    return QSIM_OK;
}

int qsim_norm(const qsim_state *st, double *norm) {
    if (int rc = check_state(st)) return rc;
    if (int rc = launch_reduce(nullptr, st->amps, st->M, st->prec, st->scratch, st->scratch_blocks, st->stream))
        return rc;
    double r[3];
    QS_CUDA(cudaMemcpyAsync(r, st->scratch + 3 * size_t(st->scratch_blocks), sizeof(r), cudaMemcpyDeviceToHost,
                            st->stream));
    QS_CUDA(cudaStreamSynchronize(st->stream));
    if (norm) *norm = r[0];
    return QSIM_OK;
}

int qsim_probabilities(const qsim_state *st, void *out, int on_device) {
    if (int rc = check_state(st)) return rc;
    if (!out) { set_error("out is NULL"); return QSIM_EINVAL; }
    const size_t n = size_t(1) << st->M;
    const size_t pb = st->prec == QSIM_C64 ? sizeof(float) : sizeof(double);
    if (on_device) return launch_probabilities(st->amps, st->M, st->prec, out, st->stream);
    void *tmp = nullptr;
    if (int rc = dmalloc(st->alloc, &tmp, n * pb, st->stream, "probabilities")) return rc;
    int rc = launch_probabilities(st->amps, st->M, st->prec, tmp, st->stream);
    if (rc == QSIM_OK) {
        cudaError_t e = cudaMemcpyAsync(out, tmp, n * pb, cudaMemcpyDeviceToHost, st->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "probabilities copy");
    }
    cudaStreamSynchronize(st->stream);
    dfree(st->alloc, tmp, n * pb, st->stream);
    return rc;
}

}  // extern "C"
