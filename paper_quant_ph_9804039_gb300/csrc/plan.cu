// Circuit plans: gate checking, grouping into passes, execution (optionally
// replayed from a captured CUDA graph).
//
// The grouping keeps the circuit's meaning: a gate is moved ahead of an
// earlier gate only when the two commute because every qubit they share is
// acted on diagonally by both (controls, and diagonal gates, are diagonal on
// their qubits).  Gate g is "blocked" once an earlier gate that shares a
// non-diagonal qubit with it has been left for a later pass.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cx.cuh"
#include "qsim_internal.h"

namespace qs {

enum StepType { S_GATE = 0, S_TILE = 1, S_FUSED = 2 };

struct Step {
    StepType type;
    Gate g;          // S_GATE
    TilePassDesc d;  // S_TILE
    double bytes;
};

}  // namespace qs

using namespace qs;

struct qsim_plan {
    int M;
    qsim_prec prec;
    qsim_opts opts;
    int mode;
    int tile_bits;
    std::vector<Gate> gates;
    std::vector<Step> steps;
    void *d_ops = nullptr;
    size_t ops_bytes = 0;
    qsim_plan_stats stats{};
    // CUDA graph of the launches for one (dst, src, stream)
    mutable cudaGraphExec_t gexec = nullptr;
    mutable void *g_dst = nullptr;
    mutable const void *g_src = nullptr;
    mutable cudaStream_t g_stream = nullptr;
    // per-launch timing
    int timing = 0;
    mutable std::vector<cudaEvent_t> ev_pool;
    mutable size_t ev_used = 0;
    mutable int64_t timed_execs = 0;
};

namespace {

inline uint64_t bit(int q) { return uint64_t(1) << q; }

int default_tile_bits(qsim_prec prec) { return prec == QSIM_C64 ? 12 : 11; }

template <typename T2>
TileOp<T2> make_tile_op(const Gate &g, const int *loc, uint64_t S) {
    TileOp<T2> op{};
    using R = decltype(T2{}.x);
    for (int k = 0; k < 4; ++k) {
        if constexpr (sizeof(R) == 4) {
            float hr, lr, hi, li;
            split_f(g.U[2 * k], hr, lr);
            split_f(g.U[2 * k + 1], hi, li);
            op.u[k] = mk(hr, hi);
            op.ul[k] = mk(lr, li);
        } else {
            op.u[k] = mk(R(g.U[2 * k]), R(g.U[2 * k + 1]));
            op.ul[k] = mk(R(0), R(0));
        }
    }
    for (int c = 0; c < g.nc; ++c) {
        if (S & bit(g.c[c]))
            op.lmask |= 1u << loc[g.c[c]];
        else
            op.gmask |= bit(g.c[c]);
    }
    if (S & bit(g.t)) {
        op.kind = g.kind;
        op.tl = uint32_t(loc[g.t]);
    } else {  // diagonal gate on a qubit outside the tile: one factor per tile
        op.kind = K_SCALE;
        if (g.kind == K_PHASE1) {  // only tiles with the target bit set change
            op.gmask |= bit(g.t);
            op.gsel = 0;
            op.u[0] = op.u[3];
            op.ul[0] = op.ul[3];
        } else {
            op.gsel = bit(g.t);
        }
    }
    return op;
}

// Greedy grouping of the gates into tile passes of at most 2^b amplitudes.
template <typename T2>
void plan_tiled(qsim_plan *p, int b_req, std::vector<TileOp<T2>> &ops) {
    const int M = p->M;
    const int b = std::min(b_req, M);
    const int L = std::min(b, p->prec == QSIM_C64 ? 5 : 4);
    const int cap = std::min(b - L, kMaxTileHigh);
    std::vector<int> rem(p->gates.size());
    for (size_t i = 0; i < rem.size(); ++i) rem[i] = int(i);
    while (!rem.empty()) {
        uint64_t defN = 0, defA = 0, high = 0;
        int nh = 0;
        std::vector<int> take, keep;
        for (int gi : rem) {
            const Gate &g = p->gates[gi];
            const uint64_t N = g.nondiag() ? bit(g.t) : 0;
            const uint64_t A = bit(g.t) | g.cmask;
            bool ok = !((N & defA) || (A & defN));
            if (ok && g.nondiag() && g.t >= L && !(high & bit(g.t))) {
                if (nh < cap) {
                    high |= bit(g.t);
                    ++nh;
                } else {
                    ok = false;
                }
            }
            if (ok) {
                take.push_back(gi);
            } else {
                keep.push_back(gi);
                defN |= N;
                defA |= A;
            }
        }
        for (int q = L; q < M && nh < cap; ++q)  // fill the tile with the lowest free qubits
            if (!(high & bit(q))) {
                high |= bit(q);
                ++nh;
            }
        const uint64_t S = (bit(L) - 1) | high;
        Step st{};
        st.type = S_TILE;
        TilePassDesc &d = st.d;
        int loc[64];
        for (int q = 0; q < 64; ++q) loc[q] = -1;
        d.L = 0;
        while (d.L < M && (S & bit(d.L))) {
            loc[d.L] = d.L;
            ++d.L;
        }
        d.nh = 0;
        d.nout = 0;
        for (int q = d.L; q < M; ++q) {
            if (S & bit(q)) {
                loc[q] = d.L + d.nh;
                d.hpos[d.nh++] = q;
            } else {
                d.opos[d.nout++] = q;
            }
        }
        d.b = d.L + d.nh;
        d.op_begin = int(ops.size());
        d.op_count = int(take.size());
        for (int gi : take) ops.push_back(make_tile_op<T2>(p->gates[gi], loc, S));
        st.bytes = 2.0 * std::ldexp(1.0, M) * double(amp_bytes(p->prec));
        p->steps.push_back(st);
        rem.swap(keep);
    }
}

int next_event(const qsim_plan *p, cudaStream_t s) {
    if (p->ev_used == p->ev_pool.size()) {
        cudaEvent_t e;
        QS_CUDA(cudaEventCreate(&e));
        p->ev_pool.push_back(e);
    }
    QS_CUDA(cudaEventRecord(p->ev_pool[p->ev_used++], s));
    return QSIM_OK;
}

int run_steps(const qsim_plan *p, void *dst, const void *src, cudaStream_t s, bool timed) {
    const size_t vec_bytes = (size_t(1) << p->M) * amp_bytes(p->prec);
    bool first = true;
    if (timed) {
        if (int rc = next_event(p, s)) return rc;
        ++p->timed_execs;
    }
    for (const Step &st : p->steps) {
        if (timed && !first)
            if (int rc = next_event(p, s)) return rc;
        if (st.type == S_TILE) {
            if (int rc = launch_tile_pass(dst, first ? src : dst, p->M, p->prec, st.d, p->d_ops, s)) return rc;
        } else {
            if (first && src != dst) QS_CUDA(cudaMemcpyAsync(dst, src, vec_bytes, cudaMemcpyDeviceToDevice, s));
            if (int rc = launch_gate(dst, p->M, p->prec, st.g, s)) return rc;
        }
        first = false;
    }
    if (first && src != dst) QS_CUDA(cudaMemcpyAsync(dst, src, vec_bytes, cudaMemcpyDeviceToDevice, s));
    if (timed && !p->steps.empty())
        if (int rc = next_event(p, s)) return rc;
    return QSIM_OK;
}

}  // namespace

extern "C" {

int qsim_plan_create(int M, qsim_prec prec, const qsim_gate *gates, size_t n, const qsim_opts *opts,
                     qsim_plan **out) {
    if (!out) { set_error("out is NULL"); return QSIM_EINVAL; }
    if (M < 1 || M > QSIM_MAX_QUBITS) { set_error("M = %d outside [1, %d]", M, QSIM_MAX_QUBITS); return QSIM_EINVAL; }
    if (prec != QSIM_C64 && prec != QSIM_C128) { set_error("unknown precision %d", int(prec)); return QSIM_EINVAL; }
    if (n > 0 && !gates) { set_error("gates is NULL"); return QSIM_EINVAL; }
    qsim_opts o{};
    if (opts) o = *opts;
    if (o.mode < QSIM_MODE_AUTO || o.mode > QSIM_MODE_FUSED) { set_error("unknown mode %d", o.mode); return QSIM_EINVAL; }
    if (o.tile_bits != 0 && (o.tile_bits < 6 || o.tile_bits > tile_max_bits(prec))) {
        set_error("tile_bits %d outside [6, %d]", o.tile_bits, tile_max_bits(prec));
        return QSIM_EINVAL;
    }
    qsim_plan *p = new qsim_plan();
    p->M = M;
    p->prec = prec;
    p->opts = o;
    p->gates.resize(n);
    for (size_t i = 0; i < n; ++i) {
        int rc = make_gate(M, gates[i].U, gates[i].target, gates[i].controls, gates[i].ncontrols, &p->gates[i]);
        if (rc) {
            char msg[512];
            snprintf(msg, sizeof msg, "gate %zu: %s", i, qsim_last_error());
            set_error("%s", msg);
            delete p;
            return rc;
        }
    }
    int mode = o.mode == QSIM_MODE_AUTO ? QSIM_MODE_TILED : o.mode;
    if (mode == QSIM_MODE_FUSED) {
        set_error("fused mode is not available in this build");
        delete p;
        return QSIM_EUNSUPPORTED;
    }
    p->mode = mode;
    const size_t ab = amp_bytes(prec);
    double bytes = 0;
    if (mode == QSIM_MODE_UNFUSED) {
        for (const Gate &g : p->gates) {
            Step st{};
            st.type = S_GATE;
            st.g = g;
            st.bytes = gate_bytes(g, M, ab);
            p->steps.push_back(st);
        }
    } else {
        const int b = o.tile_bits ? o.tile_bits : default_tile_bits(prec);
        p->tile_bits = std::min(b, M);
        int rc = tile_prepare(prec);
        if (rc == QSIM_OK) {
            if (prec == QSIM_C64) {
                std::vector<TileOp<float2>> ops;
                plan_tiled(p, b, ops);
                p->ops_bytes = ops.size() * sizeof(ops[0]);
                if (!ops.empty()) {
                    cudaError_t e = cudaMalloc(&p->d_ops, p->ops_bytes);
                    if (e == cudaSuccess) e = cudaMemcpy(p->d_ops, ops.data(), p->ops_bytes, cudaMemcpyHostToDevice);
                    if (e != cudaSuccess) rc = cuda_fail(e, "plan table upload");
                }
            } else {
                std::vector<TileOp<double2>> ops;
                plan_tiled(p, b, ops);
                p->ops_bytes = ops.size() * sizeof(ops[0]);
                if (!ops.empty()) {
                    cudaError_t e = cudaMalloc(&p->d_ops, p->ops_bytes);
                    if (e == cudaSuccess) e = cudaMemcpy(p->d_ops, ops.data(), p->ops_bytes, cudaMemcpyHostToDevice);
                    if (e != cudaSuccess) rc = cuda_fail(e, "plan table upload");
                }
            }
        }
        if (rc) {
            qsim_plan_destroy(p);
            return rc;
        }
    }
    for (const Step &st : p->steps) bytes += st.bytes;
    qsim_plan_stats &s = p->stats;
    s.n_gates = int64_t(n);
    s.n_passes = int64_t(p->steps.size());
    s.n_launches = int64_t(p->steps.size());
    s.mode = mode;
    s.tile_bits = mode == QSIM_MODE_TILED ? p->tile_bits : 0;
    s.fuse_k = 0;
    s.n_blocks = 0;
    s.algo_bytes = bytes;
    s.amp_updates = double(n) * std::ldexp(1.0, M);
    *out = p;
    return QSIM_OK;
}

int qsim_plan_execute(const qsim_plan *p, qsim_state *dst, const qsim_state *src) {
    if (!p || !dst) { set_error("plan or state is NULL"); return QSIM_EINVAL; }
    if (!src) src = dst;
    if (dst->M != p->M || dst->prec != p->prec || src->M != p->M || src->prec != p->prec) {
        set_error("state (M=%d) does not match the plan (M=%d)", dst->M, p->M);
        return QSIM_EINVAL;
    }
    cudaStream_t s = dst->stream;
    if (src != dst && src->stream != s) {
        QS_CUDA(cudaEventRecord(src->ev, src->stream));
        QS_CUDA(cudaStreamWaitEvent(s, src->ev, 0));
    }
    if (p->opts.use_graph && s != nullptr) {
        if (!(p->gexec && p->g_dst == dst->amps && p->g_src == src->amps && p->g_stream == s)) {
            if (p->gexec) {
                cudaGraphExecDestroy(p->gexec);
                p->gexec = nullptr;
            }
            QS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            int rc = run_steps(p, dst->amps, src->amps, s, false);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return cuda_fail(e, "graph capture");
            e = cudaGraphInstantiate(&p->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
            p->g_dst = dst->amps;
            p->g_src = src->amps;
            p->g_stream = s;
        }
        QS_CUDA(cudaGraphLaunch(p->gexec, s));
        return QSIM_OK;
    }
    return run_steps(p, dst->amps, src->amps, s, p->timing != 0);
}

int qsim_plan_set_timing(qsim_plan *p, int enable) {
    if (!p) { set_error("plan is NULL"); return QSIM_EINVAL; }
    p->timing = enable != 0;
    return QSIM_OK;
}

int qsim_plan_timing(qsim_plan *p, int64_t n_max, double *ms, double *bytes, int32_t *kind, int64_t *executions) {
    if (!p) { set_error("plan is NULL"); return QSIM_EINVAL; }
    const size_t nst = p->steps.size();
    const int64_t n = std::min<int64_t>(n_max, int64_t(nst));
    for (int64_t j = 0; j < n; ++j) {
        if (ms) ms[j] = 0.0;
        if (bytes) bytes[j] = p->steps[j].bytes;
        if (kind) kind[j] = int32_t(p->steps[j].type);
    }
    if (p->ev_used > 0) {
        QS_CUDA(cudaEventSynchronize(p->ev_pool[p->ev_used - 1]));
        const size_t per = nst + 1;
        for (size_t e = 0; e + per <= p->ev_used; e += per) {
            for (int64_t j = 0; j < n; ++j) {
                float t = 0.f;
                QS_CUDA(cudaEventElapsedTime(&t, p->ev_pool[e + j], p->ev_pool[e + j + 1]));
                if (ms) ms[j] += t;
            }
        }
    }
    if (executions) *executions = p->timed_execs;
    p->ev_used = 0;
    p->timed_execs = 0;
    return QSIM_OK;
}

int qsim_plan_stats_get(const qsim_plan *p, qsim_plan_stats *out) {
    if (!p || !out) { set_error("plan or out is NULL"); return QSIM_EINVAL; }
    *out = p->stats;
    return QSIM_OK;
}

void qsim_plan_destroy(qsim_plan *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    if (p->d_ops) cudaFree(p->d_ops);
    delete p;
}

int qsim_apply_circuit(qsim_state *st, const qsim_gate *gates, size_t n, const qsim_opts *opts) {
    if (!st) { set_error("state is NULL"); return QSIM_EINVAL; }
    qsim_plan *p = nullptr;
    if (int rc = qsim_plan_create(st->M, st->prec, gates, n, opts, &p)) return rc;
    int rc = qsim_plan_execute(p, st, nullptr);
    if (rc == QSIM_OK) {
        cudaError_t e = cudaStreamSynchronize(st->stream);  // the plan's tables must outlive the launches
        if (e != cudaSuccess) rc = cuda_fail(e, "circuit execution");
    }
    qsim_plan_destroy(p);
    return rc;
}

}  // extern "C"
