// A state split over P = 2^n_global ranks (Section 3.1, Section 3.3,
// Figure 8): the values of n_global "parallel" qubits select the rank that
// holds an amplitude, so every rank holds 2^(M - n_global) amplitudes and
// runs, on its own, every gate whose target is one of its local qubits.
//
// Layout: logical qubit q sits in slot slot_of[q]; slots 0 .. L-1 (L = M -
// n_global) are the bits of the local index, slot L + j is bit j of the rank.
// Initially slot_of[q] = q.  For rank r a gate becomes:
//   - a control in a global slot: the rank's bit decides; 0 leaves the gate
//     out on this rank, 1 drops the control;
//   - a diagonal gate on a global target: the factor U00 or U11 of the rank's
//     bit, applied to the local amplitudes whose (local) controls are 1;
//   - any other gate on a global target needs a redistribution first (Figure
//     8): the target is exchanged with the local qubit whose next use as such
//     a target lies furthest ahead.  The choice depends on the circuit only,
//     so every rank makes the same one.
// A redistribution of n_c pairs (global bit j_i, local slot l_i) first moves
// the l_i to the top n_c local slots (a local permutation, as SWAP gates),
// so that the amplitudes with a given value b of those bits form one
// contiguous chunk of 2^(L - n_c); rank r then swaps chunk b with the rank
// whose bits j_i are b (its chunk indexed by r's bits j_i), for every b but
// its own, and the exchanged qubits trade slots.  A fraction 1 - 2^-n_c of
// each shard moves, the factor (s^n_l - s^(n_l - n_c)) / s^n_l of EQ 2.
// With restore_order the plan ends with the standard layout again.
//
// Host logic only: the plan is made of records; a caller runs the local
// steps (qsim plans on the shard) and carries the chunks between ranks
// (NCCL send/recv, or any other transport).
#include <algorithm>
#include <cstring>
#include <vector>

#include "qsim_internal.h"

struct qsim_shard_plan {
    int M = 0, ng = 0, L = 0, rank = 0;
    struct Step {
        int kind = 0;                 // 0 local gates, 1 chunk exchange
        std::vector<qsim_gate> gates;
        std::vector<int> gbits;       // exchange: global bit of pair i (local slot L - n_c + i)
    };
    std::vector<Step> steps;
    int64_t exchanges = 0;
    double moved = 0;  // sum over exchanges of the fraction of a shard sent
};

namespace {

using qs::Gate;

qsim_gate record(const double *U, int t, int nc, const int *c) {
    qsim_gate g{};
    std::memcpy(g.U, U, sizeof g.U);
    g.target = t;
    g.ncontrols = nc;
    for (int k = 0; k < nc; ++k) g.controls[k] = c[k];
    return g;
}

void add_local(qsim_shard_plan *p, const qsim_gate &g) {
    if (p->steps.empty() || p->steps.back().kind != 0) p->steps.emplace_back();
    p->steps.back().gates.push_back(g);
}

// SWAP of two local slots as three CNOTs
void add_swap(qsim_shard_plan *p, int a, int b) {
    static const double X[8] = {0, 0, 1, 0, 1, 0, 0, 0};
    int c;
    c = a; add_local(p, record(X, b, 1, &c));
    c = b; add_local(p, record(X, a, 1, &c));
    c = a; add_local(p, record(X, b, 1, &c));
}

// Redistribution: pairs (global bit j_i, local qubit moving out into it).
void exchange(qsim_shard_plan *p, std::vector<int> &slot_of, std::vector<int> &at_slot,
              const std::vector<std::pair<int, int>> &pairs) {
    const int L = p->L, nc = int(pairs.size());
    // local permutation: the qubits moving out go to the top nc local slots
    for (int i = 0; i < nc; ++i) {
        const int want = L - nc + i;           // slot for the i-th qubit moving out
        const int q = pairs[i].second;          // the local qubit chosen to move out
        const int s = slot_of[q];
        if (s != want) {
            add_swap(p, s, want);
            const int other = at_slot[want];
            std::swap(at_slot[s], at_slot[want]);
            slot_of[q] = want;
            slot_of[other] = s;
        }
    }
    qsim_shard_plan::Step st;
    st.kind = 1;
    for (int i = 0; i < nc; ++i) {
        st.gbits.push_back(pairs[i].first);
        const int gs = L + pairs[i].first, ls = L - nc + i;
        const int qg = at_slot[gs], ql = at_slot[ls];
        std::swap(at_slot[gs], at_slot[ls]);
        slot_of[qg] = ls;
        slot_of[ql] = gs;
    }
    p->steps.push_back(st);
    ++p->exchanges;
    p->moved += 1.0 - std::ldexp(1.0, -nc);
}

}  // namespace

extern "C" {

int qsim_shard_plan_create(int M, int n_global, int rank, const qsim_gate *gates, size_t n, int restore_order,
                           qsim_shard_plan **out) {
    using namespace qs;
    if (!out) { set_error("out is NULL"); return QSIM_EINVAL; }
    if (M < 2 || M > 64) { set_error("M = %d outside [2, 64]", M); return QSIM_EINVAL; }
    if (n_global < 0 || n_global >= M || n_global > 20) {
        set_error("n_global = %d outside [0, min(M - 1, 20)]", n_global);
        return QSIM_EINVAL;
    }
    if (rank < 0 || rank >= (1 << n_global)) { set_error("rank %d outside [0, 2^%d)", rank, n_global); return QSIM_EINVAL; }
    if (n > 0 && !gates) { set_error("gates is NULL"); return QSIM_EINVAL; }
    std::vector<Gate> g(n);
    for (size_t i = 0; i < n; ++i)
        if (int rc = make_gate(M, gates[i].U, gates[i].target, gates[i].controls, gates[i].ncontrols, &g[i])) {
            char msg[512];
            snprintf(msg, sizeof msg, "gate %zu: %s", i, qsim_last_error());
            set_error("%s", msg);
            return rc;
        }
    qsim_shard_plan *p = new qsim_shard_plan();
    p->M = M;
    p->ng = n_global;
    p->L = M - n_global;
    p->rank = rank;
    const int L = p->L;
    std::vector<int> slot_of(M), at_slot(M);
    for (int q = 0; q < M; ++q) slot_of[q] = at_slot[q] = q;
    // next use of each qubit as a non-diagonal target, from gate i on
    std::vector<std::vector<size_t>> uses(M);
    for (size_t i = 0; i < n; ++i)
        if (g[i].nondiag()) uses[g[i].t].push_back(i);
    std::vector<size_t> cursor(M, 0);
    auto next_use = [&](int q, size_t i) -> size_t {
        while (cursor[q] < uses[q].size() && uses[q][cursor[q]] < i) ++cursor[q];
        return cursor[q] < uses[q].size() ? uses[q][cursor[q]] : SIZE_MAX;
    };
    for (size_t i = 0; i < n; ++i) {
        const Gate &x = g[i];
        const bool diag = !x.nondiag();
        if (!diag && slot_of[x.t] >= L) {  // redistribute: bring the target in
            int victim = -1;
            size_t far = 0;
            for (int s = 0; s < L; ++s) {
                const int q = at_slot[s];
                bool used_now = false;
                for (int c = 0; c < x.nc; ++c) used_now = used_now || x.c[c] == q;
                if (used_now) continue;  // keep this gate's local controls local
                const size_t u = next_use(q, i);
                if (victim < 0 || u > far) {
                    victim = q;
                    far = u;
                }
            }
            if (victim < 0) victim = at_slot[0];
            exchange(p, slot_of, at_slot, {{slot_of[x.t] - L, victim}});
        }
        bool live = true;
        int lc[2], nlc = 0;
        for (int c = 0; c < x.nc; ++c) {
            const int s = slot_of[x.c[c]];
            if (s >= L) live = live && ((rank >> (s - L)) & 1);
            else lc[nlc++] = s;
        }
        if (!live) continue;
        const int ts = slot_of[x.t];
        if (ts >= L) {  // diagonal gate on a global target: the rank's factor
            const int b = (rank >> (ts - L)) & 1;
            const double *f = x.U + (b ? 6 : 0);
            if (f[0] == 1.0 && f[1] == 0.0) continue;
            if (nlc == 0) {
                const double D[8] = {f[0], f[1], 0, 0, 0, 0, f[0], f[1]};
                add_local(p, record(D, 0, 0, lc));
            } else {
                const double D[8] = {1, 0, 0, 0, 0, 0, f[0], f[1]};
                add_local(p, record(D, lc[0], nlc - 1, lc + 1));
            }
            continue;
        }
        add_local(p, record(x.U, ts, nlc, lc));
    }
    if (restore_order) {
        for (;;) {  // global bit j must hold qubit L + j
            std::vector<std::pair<int, int>> pairs;
            for (int j = 0; j < n_global; ++j)
                if (at_slot[L + j] != L + j && slot_of[L + j] < L) pairs.push_back({j, L + j});
            if (!pairs.empty()) {
                exchange(p, slot_of, at_slot, pairs);
                continue;
            }
            int j = 0;
            while (j < n_global && at_slot[L + j] == L + j) ++j;
            if (j == n_global) break;
            // qubit L + j sits in another global bit: move bit j's qubit out first
            exchange(p, slot_of, at_slot, {{j, at_slot[0]}});
        }
        for (int s = 0; s < L; ++s)  // local order by selection: slot s gets qubit s
            if (at_slot[s] != s) {
                const int from = slot_of[s];
                add_swap(p, s, from);
                const int other = at_slot[s];
                std::swap(at_slot[s], at_slot[from]);
                slot_of[s] = s;
                slot_of[other] = from;
            }
    }
    *out = p;
    return QSIM_OK;
}

int qsim_shard_plan_info(const qsim_shard_plan *p, int64_t *n_steps, int64_t *n_exchanges, double *moved) {
    if (!p) { qs::set_error("plan is NULL"); return QSIM_EINVAL; }
    if (n_steps) *n_steps = int64_t(p->steps.size());
    if (n_exchanges) *n_exchanges = p->exchanges;
    if (moved) *moved = p->moved;
    return QSIM_OK;
}

int qsim_shard_step(const qsim_shard_plan *p, int64_t i, int *kind, int64_t *n_gates, int *n_pairs,
                    int *global_bits) {
    if (!p || i < 0 || i >= int64_t(p->steps.size())) { qs::set_error("no step %lld", (long long)i); return QSIM_EINVAL; }
    const qsim_shard_plan::Step &st = p->steps[size_t(i)];
    if (kind) *kind = st.kind;
    if (n_gates) *n_gates = int64_t(st.gates.size());
    if (n_pairs) *n_pairs = int(st.gbits.size());
    if (global_bits)
        for (size_t k = 0; k < st.gbits.size(); ++k) global_bits[k] = st.gbits[k];
    return QSIM_OK;
}

int qsim_shard_step_gates(const qsim_shard_plan *p, int64_t i, qsim_gate *out, size_t cap) {
    if (!p || i < 0 || i >= int64_t(p->steps.size())) { qs::set_error("no step %lld", (long long)i); return QSIM_EINVAL; }
    const qsim_shard_plan::Step &st = p->steps[size_t(i)];
    if (cap < st.gates.size() || (!out && !st.gates.empty())) {
        qs::set_error("step %lld has %zu gates, the buffer %zu", (long long)i, st.gates.size(), cap);
        return QSIM_EINVAL;
    }
    if (!st.gates.empty()) std::memcpy(out, st.gates.data(), st.gates.size() * sizeof(qsim_gate));
    return QSIM_OK;
}

void qsim_shard_plan_destroy(qsim_shard_plan *p) { delete p; }

}  // extern "C"
