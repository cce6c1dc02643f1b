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
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_fp16.h>

#include "cx.cuh"
#include "qsim_internal.h"

namespace qs {

enum StepType { S_GATE = 0, S_TILE = 1, S_FUSED = 2, S_PERM = 3 };

struct Step {
    StepType type;
    Gate g;          // S_GATE
    TilePassDesc d;  // S_TILE
    FusedDesc f;     // S_FUSED
    size_t rimg;     // S_FUSED: float offset of the block's R image
    PermDesc perm;   // S_PERM
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
    void *d_runs = nullptr;  // phase-run records of the tile passes
    size_t runs_bytes = 0;
    void *d_rimg = nullptr;  // R_hi / R_lo images of the fused blocks
    size_t rimg_bytes = 0;
    void *d_regops = nullptr;  // register-round ops and rounds of the complex64 tile passes
    size_t regops_bytes = 0;
    void *d_rounds = nullptr;
    size_t rounds_bytes = 0;
    std::vector<RegOp> h_regops;  // host copies, for qsim_plan_describe
    std::vector<RoundDesc> h_rounds;
    // specialised register passes (qsim_opts.specialize): one kernel per step, or null
    std::vector<cudaLibrary_t> jit_libs;
    std::vector<cudaKernel_t> jit_k;
    // swap runs moved to the front (step 0 permutes by front_perm); with
    // jit_gather_k the first tile pass applies it while reading a separate source
    std::vector<int> front_perm;
    cudaKernel_t jit_gather_k = nullptr;
    mutable bool last_absorbed = false;  // the last execution left the permutation pass to the gather
    std::string jit_log;
    std::string auto_log;  // the AUTO mode's estimates
    std::string group_log;  // how the fused blocks were grouped
    int *d_status = nullptr;  // set by a kernel whose bounded wait ran out
    int fuse_k = 0;
    // non-null: device tables are allocated and freed stream-ordered on this
    // stream (the serving loop), so creating and releasing a plan never
    // synchronises the device
    cudaStream_t alloc_stream = nullptr;
    DevAllocator alloc{};  // device-memory functions in force when the plan was created
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
    // touched-qubit subspace (qsim_opts.subspace): the circuit from |0...0>
    // runs as segments, each a child plan on the 2^seg_M[i] amplitudes of the
    // vector's prefix, then `relabel` moves the touched qubits from the order
    // in which they were first touched to their own positions
    bool subspace = false;
    std::vector<qsim_plan *> seg_plans;
    std::vector<int> seg_M;
    qsim_plan *relabel = nullptr;
    std::vector<int> sub_order;      // physical qubits in the order first touched
    int64_t sub_skipped = 0;         // gates left out (a control never touched)
    double sub_amp_updates = 0;      // sum over segments of gates x 2^seg_M
};

namespace {

inline uint64_t bit(int q) { return uint64_t(1) << q; }

int default_tile_bits(qsim_prec prec) { return prec == QSIM_C64 ? 12 : 11; }

// Enumeration spec: the amplitudes (diagonal kinds) or pairs (pair kinds) an
// op touches are the tile indices with the listed bits inserted.
template <typename T2>
void set_enum(TileOp<T2> &op, int tpos, bool t_insert, bool t_value, uint32_t lmask) {
    int pos[4], val[4], n = 0;
    if (t_insert) {
        pos[n] = tpos;
        val[n++] = t_value ? 1 : 0;
    }
    for (int q = 0; q < 32; ++q)
        if (lmask & (1u << q)) {
            pos[n] = q;
            val[n++] = 1;
        }
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b)
            if (pos[b] < pos[a]) {
                std::swap(pos[a], pos[b]);
                std::swap(val[a], val[b]);
            }
    op.npos = uint8_t(n);
    op.posval = 0;
    for (int a = 0; a < n; ++a) {
        op.pos[a] = uint8_t(pos[a]);
        op.posval |= uint8_t(val[a] << a);
    }
}

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
        if (g.kind == K_DENSE || g.kind == K_SWAPX)
            set_enum(op, loc[g.t], true, false, op.lmask);  // pairs: target 0, controls 1
        else if (g.kind == K_PHASE1)
            set_enum(op, loc[g.t], true, true, op.lmask);  // only target-1 states change
        else
            set_enum(op, 0, false, false, op.lmask);  // K_DIAG: every state with the controls set
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
        set_enum(op, 0, false, false, op.lmask);
    }
    return op;
}

// Pre-phase table of a run of phase gates (all qubits inside the tile) that
// precedes an uncontrolled dense gate on local target tl: entry
// (idx << 1) | target bit, idx over the local bits tpos[0..tw).  FP64
// products, stored as float hi + lo (complex64) or double (complex128).
// Float parts (re, im) of a phase factor f for kernels that multiply by them
// alone (no lo part): among the floats within two ulps of f's components, the
// pair whose squared modulus is closest to |f|^2 (then the nearest).  A
// table entry is then unit-modulus to ~1e-9 instead of ~1e-7, so that
// repeated multiplications do not drift the norm; its angle moves by at most
// two ulps (~2e-7 rad), an error that is unbiased over the entries.
void unit_hi(double fr, double fi, float *re, float *im) {
    const double m2 = fr * fr + fi * fi;
    float br = float(fr), bi = float(fi);
    double bcost = std::fabs(double(br) * br + double(bi) * bi - m2);
    double bdist = (double(br) - fr) * (double(br) - fr) + (double(bi) - fi) * (double(bi) - fi);
    float cr = float(fr);
    for (int k = 0; k < 2; ++k) cr = std::nextafter(cr, -INFINITY);
    for (int a = -2; a <= 2; ++a, cr = std::nextafter(cr, INFINITY)) {
        float ci = float(fi);
        for (int k = 0; k < 2; ++k) ci = std::nextafter(ci, -INFINITY);
        for (int b = -2; b <= 2; ++b, ci = std::nextafter(ci, INFINITY)) {
            const double cost = std::fabs(double(cr) * cr + double(ci) * ci - m2);
            const double dist = (double(cr) - fr) * (double(cr) - fr) + (double(ci) - fi) * (double(ci) - fi);
            if (cost < bcost || (cost == bcost && dist < bdist)) {
                bcost = cost;
                bdist = dist;
                br = cr;
                bi = ci;
            }
        }
    }
    *re = br;
    *im = bi;
}

template <typename T2>
uint32_t add_pre_table(std::vector<unsigned char> &runs, const std::vector<Gate> &gates, const std::vector<int> &run,
                       const int *loc, int tl, const int *tpos, int tw, bool *one0) {
    const int ne = 1 << (tw + 1);
    const size_t esz = sizeof(T2) == 8 ? 16 : 16;
    const size_t start = (runs.size() + 15) & ~size_t(15);
    runs.resize(start + size_t(ne) * esz, 0);
    *one0 = true;
    for (int e = 0; e < ne; ++e) {
        uint32_t lb = (e & 1) ? (1u << tl) : 0u;  // local bits of this entry
        for (int k = 0; k < tw; ++k)
            if ((e >> (k + 1)) & 1) lb |= 1u << tpos[k];
        double fr = 1.0, fi = 0.0;
        for (int gi : run) {
            const Gate &g = gates[gi];
            bool on = true;
            for (int c = 0; c < g.nc; ++c) on = on && ((lb >> loc[g.c[c]]) & 1);
            if (!on) continue;
            const bool up = (lb >> loc[g.t]) & 1;
            const double ur = up ? g.U[6] : g.U[0], ui = up ? g.U[7] : g.U[1];
            const double nr = fr * ur - fi * ui, ni = fr * ui + fi * ur;
            fr = nr;
            fi = ni;
        }
        if (!(e & 1) && !(fr == 1.0 && fi == 0.0)) *one0 = false;
        unsigned char *dst = runs.data() + start + size_t(e) * esz;
        if constexpr (sizeof(T2) == 8) {
            float v[4];
            unit_hi(fr, fi, &v[0], &v[1]);
            v[2] = float(fr - double(v[0]));
            v[3] = float(fi - double(v[1]));
            std::memcpy(dst, v, 16);
        } else {
            const double v[2] = {fr, fi};
            std::memcpy(dst, v, 16);
        }
    }
    return uint32_t(start);
}

constexpr int kMinPhaseRun = 6;  // shorter runs of phase gates are applied one by one

// A diagonal gate with unit-modulus entries and at most one control: its
// phase is a polynomial of degree <= 2 in the index bits.
bool is_phase_gate(const Gate &g) {
    if (!(g.kind == K_DIAG || g.kind == K_PHASE1) || g.nc > 1) return false;
    const double m0 = std::hypot(g.U[0], g.U[1]), m1 = std::hypot(g.U[6], g.U[7]);
    return std::fabs(m0 - 1.0) <= 1e-12 && std::fabs(m1 - 1.0) <= 1e-12;
}

// Angle in turns as unsigned fixed point (2^32 or 2^64 = one turn), rounded
// to nearest.
template <typename Turn>
Turn turns(double rad) {
    double t = rad / (2.0 * M_PI);
    t -= std::floor(t);  // [0, 1)
    const double hi = std::floor(t * 4294967296.0);
    if constexpr (sizeof(Turn) == 4) {
        return Turn(uint64_t(std::llround(t * 4294967296.0)) & 0xffffffffull);
    } else {
        const double lo = (t * 4294967296.0 - hi) * 4294967296.0;  // exact: t has 53 bits
        return (uint64_t(hi) << 32) + uint64_t(std::llround(lo));
    }
}

// Within one pass, move every diagonal gate as late as it can go: just before
// the first later non-diagonal gate of the pass that acts non-diagonally on
// one of its qubits (or to the end).  Diagonal gates commute with each other
// and with any gate that is diagonal on their shared qubits, so the product
// is unchanged; phase gates gathered this way form long runs.
std::vector<int> schedule_pass(const std::vector<int> &take, const std::vector<Gate> &gates) {
    std::vector<int> nd;  // positions (in take) of the non-diagonal gates
    for (size_t i = 0; i < take.size(); ++i)
        if (gates[take[i]].nondiag()) nd.push_back(int(i));
    std::vector<std::vector<int>> slot(nd.size() + 1);
    for (size_t i = 0; i < take.size(); ++i) {
        const Gate &g = gates[take[i]];
        if (g.nondiag()) continue;
        const uint64_t A = bit(g.t) | g.cmask;
        size_t k = 0;
        while (k < nd.size() && (nd[k] < int(i) || !(bit(gates[take[nd[k]]].t) & A))) ++k;
        slot[k].push_back(take[i]);
    }
    std::vector<int> out;
    out.reserve(take.size());
    for (size_t k = 0; k <= nd.size(); ++k) {
        std::stable_partition(slot[k].begin(), slot[k].end(), [&](int gi) { return is_phase_gate(gates[gi]); });
        out.insert(out.end(), slot[k].begin(), slot[k].end());
        if (k < nd.size()) out.push_back(take[nd[k]]);
    }
    return out;
}

// Phase polynomial record of a run of phase gates (layout: PhaseRunHdr).
template <typename Turn>
size_t add_phase_run(std::vector<unsigned char> &runs, const std::vector<Gate> &gates, const std::vector<int> &run,
                     int M, const int *pos, int b) {
    std::vector<Turn> c(size_t(M) + 1, Turn(0)), w(size_t(M) * M, Turn(0));  // c[0] holds c0
    for (int gi : run) {
        const Gate &g = gates[gi];
        const double a = std::atan2(g.U[1], g.U[0]), be = std::atan2(g.U[7], g.U[6]);
        const Turn ta = turns<Turn>(a), td = turns<Turn>(be - a);
        if (g.nc == 0) {
            c[0] += ta;
            c[1 + g.t] += td;
        } else {
            const int q = g.c[0];
            c[1 + q] += ta;
            w[size_t(q) * M + g.t] += td;
            w[size_t(g.t) * M + q] += td;
        }
    }
    const size_t start = (runs.size() + 15) & ~size_t(15);
    const size_t hdr = sizeof(PhaseRunHdr) + sizeof(Turn) * (size_t(M) + 1 + size_t(M) * M);
    const size_t qoff = (hdr + 15) & ~size_t(15);
    runs.resize(start + qoff + sizeof(Turn) * (size_t(1) << b), 0);
    PhaseRunHdr h{uint32_t(M), uint32_t(b), uint32_t(qoff), 0u};
    std::memcpy(runs.data() + start, &h, sizeof h);
    std::memcpy(runs.data() + start + sizeof h, c.data(), sizeof(Turn) * c.size());
    std::memcpy(runs.data() + start + sizeof h + sizeof(Turn) * c.size(), w.data(), sizeof(Turn) * w.size());
    Turn *Q = reinterpret_cast<Turn *>(runs.data() + start + qoff);
    Q[0] = 0;
    for (uint32_t u = 1; u < (1u << b); ++u) {  // Q[u] = Q[u without its top bit] + that bit's pair terms
        const int hbit = 31 - __builtin_clz(u);
        const uint32_t prev = u ^ (1u << hbit);
        Turn v = Q[prev];
        for (int j = 0; j < hbit; ++j)
            if ((prev >> j) & 1) v += w[size_t(pos[j]) * M + pos[hbit]];
        Q[u] = v;
    }
    return start;
}

// ------------------------------------------------------- register rounds
constexpr int kMaxRegOpsPerPass = kTileOpSmemBytes / int(sizeof(RegOp));

RegOp reg_op_from(const TileOp<float2> &t) {
    RegOp r{};
    for (int k = 0; k < 4; ++k) {
        r.u[k] = t.u[k];
        r.ul[k] = t.ul[k];
    }
    r.kind = t.kind;
    r.lmask = t.lmask;
    r.gmask = t.gmask;
    r.gsel = t.gsel;
    r.tb = (t.kind == K_PHASE1 || t.kind == K_DIAG) ? (1u << t.tl) : 0u;
    if (t.kind == K_DENSE) {
        bool real = true;
        for (int k = 0; k < 4; ++k) real = real && t.u[k].y == 0.f && t.ul[k].y == 0.f;
        if (real) r.kind = K_RDENSE;
    }
    return r;
}

// Group one pass's ops into rounds of RB slot qubits (greedy, moving an op
// ahead only past ops it commutes with, as for the passes themselves).
// Appends to regops / rounds; returns false if the pass cannot use them.
bool build_rounds(const std::vector<TileOp<float2>> &ops, int op_begin, int op_count, TilePassDesc &d, int RB,
                  std::vector<RegOp> &regops, std::vector<RoundDesc> &rounds, std::vector<unsigned char> &runs) {
    struct Item {
        RegOp op;
        uint32_t N, A, tl;
    };
    const uint32_t all = (d.b >= 32) ? 0xffffffffu : ((1u << d.b) - 1);
    std::vector<Item> items;
    for (int i = op_begin; i < op_begin + op_count; ++i) {
        const TileOp<float2> &t = ops[size_t(i)];
        if (t.kind == K_DENSE && t.tab_off) {  // the phase table first, then the gate
            Item it{};
            it.op.kind = K_TAB;
            it.op.gmask = 0;
            it.op.tab_off = t.tab_off;
            it.op.tw = uint8_t(t.tw + 1);
            it.op.tpos[0] = uint8_t(t.tl);
            for (int k = 0; k < t.tw; ++k) it.op.tpos[k + 1] = t.tpos[k];
            it.op.tb = (t.tflags & 1) ? (1u << t.tl) : 0u;
            uint32_t A = 1u << t.tl;
            for (int k = 0; k < t.tw; ++k) A |= 1u << t.tpos[k];
            it.N = 0;
            it.A = A;
            items.push_back(it);
        }
        Item it{};
        it.op = reg_op_from(t);
        it.tl = t.tl;
        switch (t.kind) {
            case K_DENSE:
            case K_SWAPX:
            case K_RDENSE:
                it.N = 1u << t.tl;
                it.A = it.N | t.lmask;
                break;
            case K_PHASE1:
            case K_DIAG:
                it.N = 0;
                it.A = (1u << t.tl) | t.lmask;
                break;
            case K_SCALE:
                it.N = 0;
                it.A = t.lmask;
                break;
            default:  // K_PHRUN touches every qubit
                it.N = 0;
                it.A = all;
                break;
        }
        items.push_back(it);
    }
    if (int(items.size()) > kMaxRegOpsPerPass) return false;
    d.round_begin = int(rounds.size());
    d.op_begin = int(regops.size());
    double pscale = 1.0;  // product of the deferred Hadamard factors
    int nhad = 0;
    std::vector<int> rem(items.size());
    for (size_t i = 0; i < rem.size(); ++i) rem[i] = int(i);
    bool first = true;
    while (first || !rem.empty()) {
        first = false;
        uint32_t defN = 0, defA = 0, R = 0;
        int nR = 0;
        std::vector<int> take, keep;
        for (int ii : rem) {
            const Item &it = items[size_t(ii)];
            bool ok = !((it.N & defA) || (it.A & defN));
            if (ok && it.N && !(it.N & R)) {
                if (nR < RB) {
                    R |= it.N;
                    ++nR;
                } else {
                    ok = false;
                }
            }
            if (ok) {
                take.push_back(ii);
            } else {
                keep.push_back(ii);
                defN |= it.N;
                defA |= it.A;
            }
        }
        for (int q = d.b - 1; q >= 0 && nR < RB; --q)  // fill with the highest free tile qubits
            if (!(R & (1u << q))) {
                R |= 1u << q;
                ++nR;
            }
        RoundDesc rd{};
        int k = 0;
        int slot_of[32];
        for (int q = 0; q < 32; ++q) slot_of[q] = -1;
        for (int q = 0; q < d.b; ++q)
            if (R & (1u << q)) {
                slot_of[q] = k;
                rd.pos[k++] = uint8_t(q);
            }
        rd.op_begin = uint16_t(int(regops.size()) - d.op_begin);
        rd.op_count = uint16_t(take.size());
        const uint32_t Rmask = R;
        // slots c whose slot-qubit bits include all of m's slot bits
        auto slot_mask = [&](uint32_t m, int skip_bit) {
            uint32_t sm = 0;
            for (int c = 0; c < (1 << RB); ++c) {
                if (skip_bit >= 0 && ((c >> skip_bit) & 1)) continue;
                bool ok = true;
                for (int q = 0; q < 32; ++q)
                    if ((m & Rmask & (1u << q)) && !((c >> slot_of[q]) & 1)) ok = false;
                if (ok) sm |= 1u << c;
            }
            return uint16_t(sm);
        };
        for (int ii : take) {
            RegOp op = items[size_t(ii)].op;
            const uint32_t tbit = 1u << items[size_t(ii)].tl;
            switch (op.kind) {
                case K_DENSE:
                case K_SWAPX:
                case K_RDENSE:
                    op.k = uint8_t(slot_of[items[size_t(ii)].tl]);
                    op.smask = slot_mask(op.lmask, op.k);
                    op.nmask = op.lmask & ~Rmask;
                    break;
                case K_PHASE1:
                    op.smask = slot_mask(op.lmask | tbit, -1);
                    op.nmask = (op.lmask | tbit) & ~Rmask;
                    break;
                case K_DIAG:
                    op.smask = slot_mask(op.lmask, -1);
                    op.nmask = op.lmask & ~Rmask;
                    if (Rmask & tbit) {
                        op.tbn = 0;
                        for (int c = 0; c < (1 << RB); ++c)
                            if ((c >> slot_of[items[size_t(ii)].tl]) & 1) op.tsel |= uint16_t(1u << c);
                    } else {
                        op.tbn = tbit;
                    }
                    break;
                case K_SCALE:
                    op.smask = slot_mask(op.lmask, -1);
                    op.nmask = op.lmask & ~Rmask;
                    break;
                case K_TAB:
                    op.smask = slot_mask(op.tb, -1);
                    op.nmask = op.tb & ~Rmask;
                    break;
                default:
                    break;
            }
            if (op.kind == K_PHRUN) {  // e^{i Q(slots c)} of this round, for every slot c
                PhaseRunHdr h;
                std::memcpy(&h, runs.data() + op.gsel, sizeof h);
                const uint32_t *Q = reinterpret_cast<const uint32_t *>(runs.data() + op.gsel + h.q_offset);
                float2 f[16];
                for (int c = 0; c < (1 << RB); ++c) {
                    uint32_t dep = 0;
                    for (int k2 = 0; k2 < RB; ++k2)
                        if ((c >> k2) & 1) dep |= 1u << rd.pos[k2];
                    const double ang = 2.0 * M_PI * double(Q[dep]) / 4294967296.0;
                    unit_hi(std::cos(ang), std::sin(ang), &f[c].x, &f[c].y);
                }
                const size_t start = (runs.size() + 15) & ~size_t(15);
                runs.resize(start + sizeof(f), 0);
                std::memcpy(runs.data() + start, f, sizeof(f));
                op.tab_off = uint32_t(start);
            }
            if (op.kind == K_TAB) {
                for (int c = 0; c < (1 << RB); ++c) {
                    uint32_t e = 0;
                    for (int j = 0; j < op.tw; ++j) {
                        const int sl = slot_of[op.tpos[j]];
                        if (sl >= 0 && ((c >> sl) & 1)) e |= 1u << j;
                    }
                    op.cidx[c] = uint16_t(e);
                }
            }
            {  // dispatch code
                uint32_t all_pairs = 0, all_slots = (1u << (1 << RB)) - 1;
                if (op.kind == K_DENSE || op.kind == K_RDENSE || op.kind == K_SWAPX)
                    for (int c = 0; c < (1 << RB); ++c)
                        if (!((c >> op.k) & 1)) all_pairs |= 1u << c;
                const int partial = op.smask == all_pairs ? 0 : 4;
                // (at most 64 per pass: amplitudes grow by up to sqrt(2) per deferred factor)
                const bool had = op.kind == K_RDENSE && partial == 0 && op.nmask == 0 && op.gmask == 0 && nhad < 64 &&
                                 op.u[0].x > 0.f && op.u[1].x == op.u[0].x && op.u[2].x == op.u[0].x &&
                                 op.u[3].x == -op.u[0].x && op.ul[1].x == op.ul[0].x && op.ul[2].x == op.ul[0].x &&
                                 op.ul[3].x == -op.ul[0].x;
                if (had) {
                    pscale *= double(op.u[0].x) + double(op.ul[0].x);
                    ++nhad;
                }
                // a Hadamard with an error, O = (H + E) / sqrt 2, |E| small: the
                // sums a +- b carry H, E enters as two FMA per component (its
                // entries are ~1e-4, so their float rounding is ~1e-11 absolute)
                bool near_had = false;
                if (!had && op.kind == K_RDENSE && partial == 0 && op.nmask == 0 && op.gmask == 0 && nhad < 64) {
                    const double sgn[4] = {1.0, 1.0, 1.0, -1.0};
                    double e[4];
                    near_had = true;
                    for (int j = 0; j < 4; ++j) {
                        e[j] = (double(op.u[j].x) + double(op.ul[j].x)) * M_SQRT2 - sgn[j];
                        near_had = near_had && std::fabs(e[j]) < 1.0 / 64;
                    }
                    if (near_had) {
                        for (int j = 0; j < 4; ++j) {
                            op.u[j] = make_float2(float(e[j]), 0.f);
                            op.ul[j] = make_float2(0.f, 0.f);
                        }
                        pscale *= M_SQRT1_2;
                        ++nhad;
                    }
                }
                switch (op.kind) {
                    case K_DENSE: op.code = uint8_t(RC_DENSE + partial + op.k); break;
                    case K_RDENSE:
                        op.code = uint8_t((had ? RC_HAD : near_had ? RC_NHAD : RC_RDENSE + partial) + op.k);
                        break;
                    case K_SWAPX: op.code = uint8_t(RC_SWAP + partial + op.k); break;
                    case K_PHASE1: op.code = op.smask == all_slots ? RC_PHASE_ALL : RC_PHASE; break;
                    case K_DIAG: op.code = RC_DIAG; break;
                    case K_SCALE: op.code = RC_SCALE; break;
                    case K_TAB: op.code = RC_TAB; break;
                    default: op.code = RC_PHRUN; break;
                }
            }
            regops.push_back(op);
        }
        rounds.push_back(rd);
        rem.swap(keep);
    }
    // The first round reads device memory and the last writes it, each thread
    // at its base index with the slot bits filled in: when a slot sits on tile
    // position 0, 1 or 2 the lanes of a warp are no longer 8 consecutive
    // amplitudes apart and every access is a partial sector.  Such a round
    // gets an op-free neighbour whose slots are the top tile positions, which
    // moves the tile through shared memory instead.
    auto low_slot = [&](const RoundDesc &r) {
        for (int k = 0; k < RB; ++k)
            if (r.pos[k] < 3) return true;
        return false;
    };
    if (d.b >= RB + 3) {
        RoundDesc io{};
        for (int k = 0; k < RB; ++k) io.pos[k] = uint8_t(d.b - RB + k);
        io.op_begin = 0;
        io.op_count = 0;
        if (low_slot(rounds[size_t(d.round_begin)])) rounds.insert(rounds.begin() + d.round_begin, io);
        if (low_slot(rounds.back())) rounds.push_back(io);
    }
    d.op_count = int(regops.size()) - d.op_begin;
    d.round_count = int(rounds.size()) - d.round_begin;
    d.pscale_on = pscale != 1.0;
    d.pscale_hi = float(pscale);
    d.pscale_lo = float(pscale - double(d.pscale_hi));
    return true;
}

// An uncontrolled dense gate whose rows are real up to one phase each,
// U = diag(e^{ia}, e^{ib}) O with O real (a noisy Hadamard, a NOT with a
// phase error), becomes the real gate O followed by the diagonal phase gate;
// the pass scheduler then moves the phase gate into the next run of phase
// gates, and O costs half the arithmetic of a complex 2x2.
void split_row_phases(std::vector<Gate> &gates) {
    std::vector<Gate> out;
    out.reserve(gates.size() * 2);
    for (const Gate &g : gates) {
        if (g.kind != K_DENSE || g.nc != 0) {
            out.push_back(g);
            continue;
        }
        double ph[2];
        bool ok = true;
        for (int r = 0; r < 2 && ok; ++r) {
            const double *e0 = g.U + 4 * r, *e1 = g.U + 4 * r + 2;  // row r: (re, im) of both entries
            const double m0 = std::hypot(e0[0], e0[1]), m1 = std::hypot(e1[0], e1[1]);
            const double *big = m0 >= m1 ? e0 : e1;
            ph[r] = std::atan2(big[1], big[0]);
            // the other entry must have the same phase (or be zero): Im(e conj(big)) = 0
            const double *other = m0 >= m1 ? e1 : e0;
            const double cross = other[1] * big[0] - other[0] * big[1];
            ok = std::fabs(cross) <= 1e-14 * (m0 * m0 + m1 * m1);
        }
        if (!ok) {
            out.push_back(g);
            continue;
        }
        Gate o = g, dg = g;
        for (int r = 0; r < 2; ++r) {
            const double c = std::cos(ph[r]), sn = std::sin(ph[r]);
            for (int e = 0; e < 2; ++e) {  // O = e^{-i ph_r} row r, real
                const double re = g.U[4 * r + 2 * e], im = g.U[4 * r + 2 * e + 1];
                o.U[4 * r + 2 * e] = re * c + im * sn;
                o.U[4 * r + 2 * e + 1] = 0.0;
            }
        }
        for (int k = 0; k < 8; ++k) dg.U[k] = 0.0;
        dg.U[0] = ph[0] == 0.0 ? 1.0 : std::cos(ph[0]);
        dg.U[1] = ph[0] == 0.0 ? 0.0 : std::sin(ph[0]);
        dg.U[6] = std::cos(ph[1]);
        dg.U[7] = std::sin(ph[1]);
        dg.kind = (dg.U[0] == 1.0 && dg.U[1] == 0.0) ? K_PHASE1 : K_DIAG;
        if (ph[0] == 0.0 && ph[1] == 0.0) {
            out.push_back(o);  // already real
        } else {
            out.push_back(o);
            out.push_back(dg);
        }
    }
    gates.swap(out);
}

// Runs of SWAP gates written as three exact CNOTs (a->b, b->a, a->b).
// Returns, for every gate, -1 or the id of the run it belongs to, and the
// runs' qubit permutations (pi[q] = new position of qubit q).
int find_swap_runs(const std::vector<Gate> &g, std::vector<int> &run_of, std::vector<std::vector<int>> &perms, int M) {
    run_of.assign(g.size(), -1);
    int nrun = 0;
    size_t i = 0;
    while (i + 2 < g.size()) {
        auto is_swap = [&](size_t k) {
            const Gate &a = g[k], &b = g[k + 1], &c = g[k + 2];
            return a.kind == K_SWAPX && b.kind == K_SWAPX && c.kind == K_SWAPX && a.nc == 1 && b.nc == 1 &&
                   c.nc == 1 && a.t == c.t && a.c[0] == c.c[0] && b.t == a.c[0] && b.c[0] == a.t;
        };
        if (!is_swap(i)) {
            ++i;
            continue;
        }
        std::vector<int> pi(M);
        for (int q = 0; q < M; ++q) pi[q] = q;
        size_t j = i;
        while (j + 2 < g.size() && is_swap(j)) {
            const int a = g[j].c[0], b = g[j].t;
            for (int q = 0; q < M; ++q) {  // compose: positions a and b exchange
                if (pi[q] == a) pi[q] = b;
                else if (pi[q] == b) pi[q] = a;
            }
            for (size_t k = j; k < j + 3; ++k) run_of[k] = nrun;
            j += 3;
        }
        bool invol = true;
        for (int q = 0; q < M; ++q) invol = invol && pi[pi[q]] == q;
        if (!invol) {  // leave it as gates
            for (size_t k = i; k < j; ++k) run_of[k] = -1;
        } else {
            perms.push_back(pi);
            ++nrun;
        }
        i = j;
    }
    return nrun;
}

// The deferred Hadamard factors of the register passes (a scalar, which
// commutes with every later op and permutation) are carried forward and
// applied once, compensated, by the last register pass of the plan, instead
// of once per pass.  Amplitudes grow meanwhile; a pass applies what it
// carries as soon as the carried factor falls below 2^-24 (so a normalised
// state stays below 2^56 inside any pass).
void carry_pass_scales(std::vector<Step> &steps) {
    double carry = 1.0;
    Step *last = nullptr;
    for (Step &st : steps) {
        if (st.type != S_TILE || st.d.round_count == 0) continue;
        last = &st;
        if (st.d.pscale_on) carry *= double(st.d.pscale_hi) + double(st.d.pscale_lo);
        st.d.pscale_on = 0;
        if (carry < std::ldexp(1.0, -24)) {
            st.d.pscale_on = 1;
            st.d.pscale_hi = float(carry);
            st.d.pscale_lo = float(carry - double(st.d.pscale_hi));
            carry = 1.0;
        }
    }
    if (last && carry != 1.0) {
        last->d.pscale_on = 1;
        last->d.pscale_hi = float(carry);
        last->d.pscale_lo = float(carry - double(last->d.pscale_hi));
    }
}

// Every swap run moved to the front of the circuit.  A run that exchanges
// qubit positions (pi[q] = new position of q) can be left out if every later
// gate is relabelled instead: with phi[q] = where the data of qubit q sits,
// phi starts as the product Q of all runs applied to the input, and each run
// met on the way turns phi into phi o pi^-1, ending at the identity.  The
// gates keep their order and matrices; only their qubits move.  Taken only
// when Q is an involution (the permutation pass works in place on those).
// Returns Q, or an empty vector (nothing changed).
std::vector<int> swaps_to_front(std::vector<Gate> &gates, const std::vector<int> &run_of,
                                const std::vector<std::vector<int>> &perms, int M) {
    if (perms.empty()) return {};
    std::vector<int> Q(M);
    for (int q = 0; q < M; ++q) Q[q] = q;
    for (const std::vector<int> &pi : perms)
        for (int q = 0; q < M; ++q) Q[q] = pi[Q[q]];
    for (int q = 0; q < M; ++q)
        if (Q[Q[q]] != q) return {};
    std::vector<int> phi = Q;
    std::vector<Gate> out;
    out.reserve(gates.size());
    for (size_t gi = 0; gi < gates.size(); ++gi) {
        const int r = run_of[gi];
        if (r >= 0) {
            if (gi == 0 || run_of[gi - 1] != r) {
                std::vector<int> inv(M), nphi(M);
                for (int q = 0; q < M; ++q) inv[perms[size_t(r)][q]] = q;
                for (int q = 0; q < M; ++q) nphi[q] = phi[inv[q]];
                phi.swap(nphi);
            }
            continue;
        }
        Gate g = gates[gi];
        g.t = phi[g.t];
        g.cmask = 0;
        for (int c = 0; c < g.nc; ++c) {
            g.c[c] = phi[g.c[c]];
            g.cmask |= bit(g.c[c]);
        }
        out.push_back(g);
    }
    gates.swap(out);
    return Q;
}

// Shared-memory wavefronts of one warp access (lane byte addresses, `width`
// bytes each): the lanes are served in groups that move 128 bytes (32 lanes
// of 4-byte, 16 of 8-byte, 8 of 16-byte accesses); within a group, the
// largest number of distinct 4-byte words on one bank.
int wavefronts(const uint32_t *addr, int width) {
    const int group = width >= 16 ? 8 : (width == 8 ? 16 : 32);
    int total = 0;
    for (int g0 = 0; g0 < 32; g0 += group) {
        uint32_t words[32][64];
        int cnt[32] = {0};
        int worst = 1;
        for (int l = g0; l < g0 + group; ++l)
            for (int w = 0; w < width / 4; ++w) {
                const uint32_t word = addr[l] / 4 + uint32_t(w);
                const int bank = int(word & 31);
                bool seen = false;
                for (int i = 0; i < cnt[bank]; ++i) seen |= words[bank][i] == word;
                if (!seen) {
                    words[bank][cnt[bank]++] = word;
                    worst = std::max(worst, cnt[bank]);
                }
            }
        total += worst;
    }
    return total;
}

// Tile of the permutation pass: the lowest lb qubits (contiguous runs of
// 2^lb amplitudes) and their images under pi, with lb as large as the shared
// memory of two tiles allows (at most 12 tile qubits).
PermDesc perm_desc(const std::vector<int> &pi, int M, qsim_prec prec) {
    PermDesc best{};
    for (int lb = std::min(6, M); lb >= 1; --lb) {
        PermDesc d{};
        d.lb = lb;
        uint64_t S = 0;
        for (int q = 0; q < lb; ++q) S |= bit(q) | bit(pi[q]);
        if (__builtin_popcountll(S) > 12) continue;
        int sidx[64], oidx[64];
        for (int q = 0; q < M; ++q) {
            if (S & bit(q)) {
                sidx[q] = d.ns;
                d.spos[d.ns++] = q;
            } else {
                oidx[q] = d.nout;
                d.opos[d.nout++] = q;
            }
        }
        for (int j = 0; j < d.ns; ++j) d.spi[j] = sidx[pi[d.spos[j]]];
        for (int j = 0; j < d.nout; ++j) d.opi[j] = oidx[pi[d.opos[j]]];
        // shared-memory swizzle: fewest wavefronts over the warp writes in index
        // order and the warp reads at sig(v) (v in index order)
        const uint32_t n = 1u << d.ns;
        std::vector<uint32_t> sig(n);
        for (uint32_t u = 0; u < n; ++u) {
            uint32_t v = 0;
            for (int j = 0; j < d.ns; ++j)
                if ((u >> j) & 1) v |= 1u << d.spi[j];
            sig[u] = v;
        }
        const int ab = int(amp_bytes(prec));
        long best_cost = -1;
        for (int sh = 4; sh <= std::max(4, d.ns - 1); ++sh) {
            long cost = 0;
            uint32_t wa[32], ra[32];
            for (uint32_t w0 = 0; w0 < n; w0 += 32) {
                for (uint32_t l = 0; l < 32; ++l) {
                    const uint32_t u = (w0 + l) % n, sv = sig[u];
                    wa[l] = uint32_t(ab) * (u ^ ((u >> sh) & 15u));
                    ra[l] = uint32_t(ab) * (sv ^ ((sv >> sh) & 15u));
                }
                cost += wavefronts(wa, ab) + wavefronts(ra, ab);
            }
            if (best_cost < 0 || cost < best_cost) {
                best_cost = cost;
                d.sh = sh;
            }
        }
        if (perm_smem_bytes(d, prec) <= 96 * 1024) return d;
        best = d;
    }
    return best;
}

// Greedy grouping of the gates into tile passes of at most 2^b amplitudes.
// `reserve`: qubits that the first pass's tile holds whatever its gates (the
// source-order runs of a permutation that pass gathers).
template <typename T2>
void plan_tiled(qsim_plan *p, int b_req, std::vector<int> rem, std::vector<TileOp<T2>> &ops,
                std::vector<unsigned char> &runs, uint64_t reserve = 0) {
    const int M = p->M;
    const int b = std::min(b_req, M);
    const int L = std::min(b, p->prec == QSIM_C64 ? 5 : 4);
    const int cap = std::min(b - L, kMaxTileHigh);
    reserve &= ~(bit(L) - 1);
    if (__builtin_popcountll(reserve) > cap) reserve = 0;
    while (!rem.empty()) {
        uint64_t defN = 0, defA = 0, high = reserve;
        int nh = __builtin_popcountll(reserve);
        reserve = 0;
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
        int pos[kMaxTileHigh + 8];  // global qubit of each tile-local bit
        for (int j = 0; j < d.L; ++j) pos[j] = j;
        for (int j = 0; j < d.nh; ++j) pos[d.L + j] = d.hpos[j];
        d.op_begin = int(ops.size());
        const std::vector<int> seq = schedule_pass(take, p->gates);
        for (size_t i = 0; i < seq.size();) {
            size_t j = i;
            while (j < seq.size() && is_phase_gate(p->gates[seq[j]])) ++j;
            if (j == i) {  // a non-phase gate
                ops.push_back(make_tile_op<T2>(p->gates[seq[i]], loc, S));
                ++i;
                continue;
            }
            const std::vector<int> run(seq.begin() + i, seq.begin() + j);
            // a run followed by an uncontrolled dense gate, all inside the tile
            // and over at most 8 other local bits, rides on that gate
            if (j < seq.size() && p->gates[seq[j]].kind == K_DENSE && p->gates[seq[j]].nc == 0) {
                const int tl = loc[p->gates[seq[j]].t];
                uint32_t bits = 0;
                bool inside = true;
                for (int gi : run) {
                    const Gate &g = p->gates[gi];
                    inside = inside && (S & bit(g.t));
                    for (int c = 0; c < g.nc; ++c) inside = inside && (S & bit(g.c[c]));
                    if (!inside) break;
                    bits |= 1u << loc[g.t];
                    for (int c = 0; c < g.nc; ++c) bits |= 1u << loc[g.c[c]];
                }
                bits &= ~(1u << tl);
                if (inside && tl >= 0 && __builtin_popcount(bits) <= 8) {
                    TileOp<T2> op = make_tile_op<T2>(p->gates[seq[j]], loc, S);
                    int tpos[8], tw = 0;
                    for (int q = 0; q < 32; ++q)
                        if (bits & (1u << q)) tpos[tw++] = q;
                    bool one0 = false;
                    if (runs.empty()) runs.resize(16, 0);  // offset 0 means "no table"
                    op.tab_off = add_pre_table<T2>(runs, p->gates, run, loc, tl, tpos, tw, &one0);
                    op.tw = uint8_t(tw);
                    op.tflags = one0 ? 1 : 0;
                    for (int k = 0; k < tw; ++k) op.tpos[k] = uint8_t(tpos[k]);
                    ops.push_back(op);
                    i = j + 1;
                    continue;
                }
            }
            if (run.size() >= size_t(kMinPhaseRun)) {
                TileOp<T2> op{};
                op.kind = K_PHRUN;
                if (runs.empty()) runs.resize(16, 0);
                op.gsel = add_phase_run<TurnT<T2>>(runs, p->gates, run, M, pos, d.b);
                ops.push_back(op);
            } else {
                for (int gi : run) ops.push_back(make_tile_op<T2>(p->gates[gi], loc, S));
            }
            i = j;
        }
        d.op_count = int(ops.size()) - d.op_begin;
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

// --------------------------------------------------------------- fused mode
// Product of the block's gates (in order) as a dense 2^k x 2^k matrix, FP64:
// each gate's 2x2 operation applied to every column (Section 2.1's pair rule
// on the 2^k-dimensional block space).
std::vector<double> block_matrix(const std::vector<Gate> &gates, const std::vector<int> &take, const int *bq, int k) {
    const int n = 1 << k;
    std::vector<double> U(size_t(2) * n * n, 0.0);  // U[(row * n + col) * 2 + re/im]
    for (int i = 0; i < n; ++i) U[size_t(2) * (i * n + i)] = 1.0;
    auto local = [&](int q) {
        for (int j = 0; j < k; ++j)
            if (bq[j] == q) return j;
        return -1;
    };
    for (int gi : take) {
        const Gate &g = gates[gi];
        const int t = local(g.t);
        uint32_t cm = 0;
        for (int c = 0; c < g.nc; ++c) cm |= 1u << local(g.c[c]);
        for (int i = 0; i < n; ++i) {
            if ((i >> t) & 1 || (uint32_t(i) & cm) != cm) continue;
            const int j = i | (1 << t);
            for (int col = 0; col < n; ++col) {
                double *a = &U[size_t(2) * (i * n + col)], *b = &U[size_t(2) * (j * n + col)];
                const double ar = a[0], ai = a[1], br = b[0], bi = b[1];
                const double *u = g.U;
                a[0] = u[0] * ar - u[1] * ai + u[2] * br - u[3] * bi;
                a[1] = u[0] * ai + u[1] * ar + u[2] * bi + u[3] * br;
                b[0] = u[4] * ar - u[5] * ai + u[6] * br - u[7] * bi;
                b[1] = u[4] * ai + u[5] * ar + u[6] * bi + u[7] * br;
            }
        }
    }
    return U;
}

// U^dagger U = I to 1e-10 (FP64).
bool is_unitary(const std::vector<double> &U, int k) {
    const int n = 1 << k;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double re = 0, im = 0;
            for (int r = 0; r < n; ++r) {  // sum_r conj(U[r][i]) U[r][j]
                const double ar = U[size_t(2) * (r * n + i)], ai = U[size_t(2) * (r * n + i) + 1];
                const double br = U[size_t(2) * (r * n + j)], bi = U[size_t(2) * (r * n + j) + 1];
                re += ar * br + ai * bi;
                im += ar * bi - ai * br;
            }
            if (std::fabs(re - (i == j ? 1.0 : 0.0)) > 1e-10 || std::fabs(im) > 1e-10) return false;
        }
    return true;
}

// Shared-memory byte offset of element (row, column c) of a K-major operand
// with rows of W bytes (W = 128, 64, 32 for k = 5, 4, 3): 16-byte chunks of
// each row XOR-swizzled by the row bits above them, as the MMA descriptors of
// layout SW128 / SW64 / SW32 read them.
uint32_t operand_offset(int W, uint32_t row, uint32_t byte_in_row) {
    const uint32_t sw = W == 128 ? (row & 7) : (W == 64 ? ((row >> 1) & 3) : ((row >> 2) & 1));
    return row * uint32_t(W) ^ (sw << 4) ^ byte_in_row;
}

// R_hi and R_lo (FP16, R scaled by 2^8) of the block as the MMA's B operand:
// row n = output real, column kk = input real.
void block_rimg(const std::vector<double> &U, int k, __half *img) {
    const int n = 1 << k, KR = 2 * n, W = 2 * KR;
    const size_t plane = size_t(KR) * KR;
    for (int r = 0; r < KR; ++r) {
        for (int kk = 0; kk < KR; ++kk) {
            const int a = r >> 1, b = kk >> 1;
            const double ur = U[size_t(2) * (a * n + b)], ui = U[size_t(2) * (a * n + b) + 1];
            double v;
            if ((r & 1) == 0) v = (kk & 1) ? -ui : ur;
            else v = (kk & 1) ? ur : ui;
            v *= 256.0;
            const __half hi = __float2half_rn(float(v));
            const __half lo = __float2half_rn(float(v - double(__half2float(hi))));
            const size_t off = operand_offset(W, uint32_t(r), uint32_t(2 * kk)) / 2;
            img[off] = hi;
            img[plane + off] = lo;
        }
    }
}

// Shared-memory wavefronts of the split warps' operand writes for skew
// candidate (c, sh) of fused_desc at width k: they depend on the width only
// (not on the block's qubits), so they are counted once per process.
long operand_write_cost(int k, int c, int sh) {
    struct Table {
        long v[6][18][6];
    };
    static const Table table = [] {
        Table t{};
        for (int kk = 3; kk <= 5; ++kk) {
            const int NA = 1 << kk, W = 4 * NA, NROWS = 1 << (kFusedTileBits - kk);
            uint32_t sa[32];
            for (int cc = 0; cc < 18; ++cc)
                for (int s = 0; s < 6; ++s) {
                    long cost = 0;
                    for (int w = 0; w < 4; ++w)
                        for (int st = 0; st < NA; ++st) {
                            for (int l = 0; l < 32; ++l) {
                                const int g = ((l * (cc == 0 ? 0 : 2 * cc - 1)) ^ (s ? (l >> s) : 0)) & (NA - 1);
                                sa[l] = operand_offset(W, uint32_t(32 * w + l), 4u * uint32_t(st ^ g));
                            }
                            cost += 2 * wavefronts(sa, 4);
                        }
                    t.v[kk][cc][s] = cost * (NROWS / 128);
                }
        }
        return t;
    }();
    return table.v[k][c][sh];
}

FusedDesc fused_desc_compute(int M, int k, const int *bq) {
    FusedDesc d{};
    d.k = k;
    const int nf = kFusedTileBits - k, NA = 1 << k, NROWS = 1 << nf, KR = 2 * NA, W = 2 * KR;
    uint64_t B = 0;
    for (int j = 0; j < k; ++j) B |= bit(bq[j]);
    uint64_t F = 0;
    int fq[kFusedTileBits], nfq = 0;
    for (int q = 0; q < M && nfq < nf; ++q)
        if (!(B & bit(q))) {
            F |= bit(q);
            fq[nfq++] = q;
        }
    const uint64_t Uq = B | F;
    int idx[64];
    int nu = 0;
    for (int q = 0; q < M; ++q)
        if (Uq & bit(q)) idx[q] = nu++;
    d.runbits = 0;
    while (d.runbits < M && (Uq & bit(d.runbits))) ++d.runbits;
    d.nrb = 0;
    for (int q = d.runbits; q < M; ++q)
        if (Uq & bit(q)) d.rpos[d.nrb++] = q;
    d.nout = 0;
    for (int q = 0; q < M; ++q)
        if (!(Uq & bit(q))) d.opos[d.nout++] = q;
    for (int a = 0; a < NA; ++a) {
        uint32_t u = 0;
        for (int j = 0; j < k; ++j)
            if ((a >> j) & 1) u |= 1u << idx[bq[j]];
        d.posA[a] = uint16_t(u);
    }
    for (int m = 0; m < NROWS; ++m) {
        uint32_t u = 0;
        for (int j = 0; j < nf; ++j)
            if ((m >> j) & 1) u |= 1u << idx[fq[j]];
        d.posM[m] = uint16_t(u);
    }
    // Direct stores (each thread writes its own sub-vector row to device memory)
    // when qubits 0 and 1 are outside the block: a warp's stores of one
    // combination then fill whole 32-byte sectors (4 consecutive amplitudes).
    // Measured per block at M=28 (TB/s, staged / direct): block on qubits 0..4
    // 4.9 / 2.8, 1..5 4.9 / 4.1, 2..6 4.7 / 5.2, 3..7 4.9 / 6.0, 4..8 4.9 / 6.1.
    d.direct = 1;
    for (int m = 0; m < 4 && m < NROWS; ++m) d.direct &= d.posM[m] == m ? 1 : 0;
    for (int j = 0; j < 32; ++j) {
        const uint32_t u = uint32_t(j) << 7;
        uint64_t off = 0;
        for (int b = 7; b < kFusedTileBits; ++b)
            if ((u >> b) & 1) off |= b < d.runbits ? bit(b) : bit(d.rpos[b - d.runbits]);
        d.runoff2[j] = off;
    }
    // split: lane l of split warp w owns sub-vector rows 32 w + l (+ 128 per row
    // block) and visits combination s ^ skew[l] at step s; pick the skew with the
    // fewest shared-memory wavefronts over the warp's input reads and operand writes
    {
        long best = -1;
        uint32_t la[32];
        uint8_t g[32];
        for (int c = 0; c < 18; ++c)
            for (int sh = 0; sh < 6; ++sh) {
                for (int l = 0; l < 32; ++l) g[l] = uint8_t(((l * (c == 0 ? 0 : 2 * c - 1)) ^ (sh ? (l >> sh) : 0)) & (NA - 1));
                long cost = operand_write_cost(k, c, sh);
                for (int w = 0; w < 4; ++w)
                    for (int rb = 0; rb < NROWS / 128; ++rb)
                        for (int st = 0; st < NA; ++st) {
                            for (int l = 0; l < 32; ++l) {
                                const int rho = 32 * w + l, a = st ^ g[l];
                                la[l] = 8u * (uint32_t(d.posA[a]) | d.posM[rb * 128 + rho]);
                            }
                            cost += wavefronts(la, 8);
                        }
                if (best < 0 || cost < best) {
                    best = cost;
                    std::memcpy(d.skew, g, 32);
                }
            }
    }
    // epilogue: thread = sub-vector row, writes combination a at swz(posA[a] | posM[m]);
    // then warp w reads back the quarter of the tile whose bits posM[32],
    // posM[64] equal w, 16 bytes (an aligned pair) a lane; pick the staging
    // swizzle shift
    {
        long best = -1;
        uint32_t ad[32];
        for (int r = 4; r <= 8; ++r) {
            auto swz = [r](uint32_t u) { return u ^ ((u >> r) & 15u); };
            long cost = 0;
            for (int w = 0; w < 4; ++w)
                for (int rb = 0; rb < NROWS / 128; ++rb)
                    for (int a = 0; a < NA; ++a) {
                        for (int l = 0; l < 32; ++l) ad[l] = 8u * swz(uint32_t(d.posA[a]) | d.posM[rb * 128 + 32 * w + l]);
                        cost += wavefronts(ad, 8);
                    }
            const uint32_t b5 = d.posM[32], b6 = d.posM[64];
            for (int w = 0; w < 4; ++w)
                for (int it = 0; it < 16; ++it) {
                    for (int l = 0; l < 32; ++l) {
                        uint32_t u = uint32_t(it * 64 + 2 * l);
                        u = ((u & ~(b5 - 1u)) << 1) | (u & (b5 - 1u));
                        u = ((u & ~(b6 - 1u)) << 1) | (u & (b6 - 1u));
                        u |= ((w & 1) ? b5 : 0u) | ((w & 2) ? b6 : 0u);
                        ad[l] = 8u * (swz(u) & ~1u);
                    }
                    cost += wavefronts(ad, 16);
                }
            if (best < 0 || cost < best) {
                best = cost;
                d.outsh = r;
            }
        }
    }
    return d;
}

// fused_desc_compute is a pure function of (M, k, the block's qubits) that
// takes milliseconds (the wavefront searches): its results are kept for the
// process (at most kDescCacheMax of them), so the ideal and noisy circuits,
// and every later plan over the same qubit sets, look them up.
constexpr size_t kDescCacheMax = 4096;
std::mutex g_desc_mu;
std::map<std::pair<uint64_t, int>, FusedDesc> g_desc_cache;

std::pair<uint64_t, int> desc_key(int M, int k, const int *bq) {
    uint64_t B = 0;
    for (int j = 0; j < k; ++j) B |= bit(bq[j]);
    return {B, M * 8 + k};
}

bool desc_lookup(int M, int k, const int *bq, FusedDesc *d) {
    std::lock_guard<std::mutex> lock(g_desc_mu);
    auto it = g_desc_cache.find(desc_key(M, k, bq));
    if (it == g_desc_cache.end()) return false;
    *d = it->second;
    return true;
}

void desc_store(int M, int k, const int *bq, const FusedDesc &d) {
    std::lock_guard<std::mutex> lock(g_desc_mu);
    if (g_desc_cache.size() >= kDescCacheMax) g_desc_cache.clear();
    g_desc_cache[desc_key(M, k, bq)] = d;
}

FusedDesc fused_desc(int M, int k, const int *bq) {
    FusedDesc d;
    if (desc_lookup(M, k, bq, &d)) return d;
    d = fused_desc_compute(M, k, bq);
    desc_store(M, k, bq, d);
    return d;
}

// Grouping into blocks of k qubits (every qubit of a gate, controls
// included, belongs to the block).  A gate may join a block ahead of earlier
// gates left for later blocks only if it commutes with each of them: neither
// gate's non-diagonal target is a qubit of the other.  For each block the
// candidates are the greedy set (gates taken in order while their qubits fit,
// padded to k with the lowest free qubits) and every window of k consecutive
// qubits; the candidate that takes the most remaining gates wins (on the
// 33-qubit brickwork: 75 blocks per circuit instead of the greedy 108;
// fused_groups_beam below searches further).
struct FusedGroup {
    uint64_t Q;
    std::vector<int> take;
};
std::vector<FusedGroup> fused_groups(const std::vector<Gate> &gates, int k, int M) {
    std::vector<int> rem(gates.size());
    for (size_t i = 0; i < rem.size(); ++i) rem[i] = int(i);
    std::vector<FusedGroup> out;
    std::vector<int> take, keep, best_take, best_keep;
    while (!rem.empty()) {
        // the greedy candidate
        uint64_t defN = 0, defA = 0, Q = 0;
        take.clear();
        keep.clear();
        for (int gi : rem) {
            const Gate &g = gates[size_t(gi)];
            const uint64_t N = g.nondiag() ? bit(g.t) : 0;
            const uint64_t A = bit(g.t) | g.cmask;
            if (!((N & defA) || (A & defN)) && __builtin_popcountll(Q | A) <= k) {
                take.push_back(gi);
                Q |= A;
            } else {
                keep.push_back(gi);
                defN |= N;
                defA |= A;
            }
        }
        for (int q = 0; q < M && __builtin_popcountll(Q) < k; ++q) Q |= bit(q);
        uint64_t bestQ = Q;
        best_take.swap(take);
        best_keep.swap(keep);
        // the windows of k consecutive qubits
        for (int s = 0; s + k <= M; ++s) {
            const uint64_t W = ((uint64_t(1) << k) - 1) << s;
            defN = defA = 0;
            take.clear();
            keep.clear();
            for (int gi : rem) {
                const Gate &g = gates[size_t(gi)];
                const uint64_t N = g.nondiag() ? bit(g.t) : 0;
                const uint64_t A = bit(g.t) | g.cmask;
                if (!((N & defA) || (A & defN)) && !(A & ~W)) {
                    take.push_back(gi);
                } else {
                    keep.push_back(gi);
                    defN |= N;
                    defA |= A;
                }
            }
            if (take.size() > best_take.size()) {
                bestQ = W;
                best_take.swap(take);
                best_keep.swap(keep);
            }
        }
        out.push_back({bestQ, best_take});
        rem.swap(best_keep);
    }
    return out;
}

// fn(t) for t in [0, nt) on threads; whatever cannot get a thread runs here.
template <class F>
void run_parallel(size_t nt, F fn) {
    std::vector<std::thread> pool;
    size_t started = 0;
    try {
        for (; started < nt; ++started) pool.emplace_back(fn, started);
    } catch (...) {
    }
    for (size_t t = started; t < nt; ++t) fn(t);
    for (std::thread &th : pool) th.join();
}

// Beam search over the same candidates (every window of k consecutive
// qubits, and the greedy set): at each depth every kept partial grouping is
// extended by every candidate, extensions that leave the same gates are
// merged, and the `width` best by (cost so far + the remaining gates, a
// controlled gate counting 3, over 16) are kept.  A block costs 1, or
// search_cost when it holds qubit 0 or 1 (those blocks store through the
// staging tile and run slower).  The search is not monotone in its cost
// weight, so fused_groups_beam runs it with six weights (1, the measured
// staged/direct ratio, their mean, 1.15, 1.25 and 1.5) and keeps the grouping
// with the lowest cost at the measured ratio, or fused_groups' when that is
// cheaper (on the 33-qubit brickwork with 24 layers: 70 blocks, 8 of them
// staged, against 75 and 10).
double grouping_cost(const std::vector<FusedGroup> &g, double staged_cost) {
    double c = 0;
    for (const FusedGroup &x : g) c += (x.Q & 3u) ? staged_cost : 1.0;
    return c;
}

std::vector<FusedGroup> beam_search(const std::vector<Gate> &gates, int k, int M, int width, double staged_cost,
                                    const std::vector<FusedGroup> &base) {
    if (width < 2 || gates.empty()) return base;
    const size_t n = gates.size();
    std::vector<uint64_t> gN(n), gA(n);
    std::vector<int> gw(n);
    for (size_t i = 0; i < n; ++i) {
        gN[i] = gates[i].nondiag() ? bit(gates[i].t) : 0;
        gA[i] = bit(gates[i].t) | gates[i].cmask;
        gw[i] = gates[i].nc > 0 ? 3 : 1;
    }
    struct State {
        double cost;
        std::vector<int> rem;
        std::vector<FusedGroup> hist;
    };
    struct Child {
        double cost, score;
        int parent;
        uint64_t Q, hash;
        size_t ntake;
    };
    // one candidate block Q on a state's remaining gates: its cost, score and
    // a hash of the gates it leaves (materialised only for the kept children)
    auto scan = [&](const State &st, int parent, uint64_t Q) {
        uint64_t defN = 0, defA = 0, h = 1469598103934665603ull;
        long wsum = 0;
        size_t ntake = 0;
        for (int gi : st.rem) {
            const uint64_t N = gN[size_t(gi)], A = gA[size_t(gi)];
            if (!((N & defA) || (A & defN)) && !(A & ~Q)) {
                ++ntake;
            } else {
                defN |= N;
                defA |= A;
                wsum += gw[size_t(gi)];
                h = (h ^ uint64_t(gi)) * 1099511628211ull;
            }
        }
        Child c;
        c.parent = parent;
        c.Q = Q;
        c.ntake = ntake;
        c.hash = h ^ uint64_t(st.rem.size() - ntake);
        c.cost = st.cost + ((Q & 3u) ? staged_cost : 1.0);
        c.score = c.cost + double(wsum) / 16.0;
        return c;
    };
    auto materialise = [&](const State &st, uint64_t Q, std::vector<int> &take, std::vector<int> &keep) {
        uint64_t defN = 0, defA = 0;
        for (int gi : st.rem) {
            const uint64_t N = gN[size_t(gi)], A = gA[size_t(gi)];
            if (!((N & defA) || (A & defN)) && !(A & ~Q)) {
                take.push_back(gi);
            } else {
                keep.push_back(gi);
                defN |= N;
                defA |= A;
            }
        }
    };
    std::vector<uint64_t> windows;
    for (int s0 = 0; s0 + k <= M; ++s0) windows.push_back(((uint64_t(1) << k) - 1) << s0);
    auto greedy_set = [&](const State &st) {  // the greedy set, padded with the lowest free qubits
        uint64_t defN = 0, defA = 0, Q = 0;
        for (int gi : st.rem) {
            const uint64_t N = gN[size_t(gi)], A = gA[size_t(gi)];
            if (!((N & defA) || (A & defN)) && __builtin_popcountll(Q | A) <= k) {
                Q |= A;
            } else {
                defN |= N;
                defA |= A;
            }
        }
        for (int q = 0; q < M && __builtin_popcountll(Q) < k; ++q) Q |= bit(q);
        return Q;
    };
    std::vector<State> beam(1);
    beam[0].cost = 0;
    beam[0].rem.resize(n);
    for (size_t i = 0; i < n; ++i) beam[0].rem[i] = int(i);
    std::vector<Child> all;
    for (size_t depth = 0; depth <= n; ++depth) {
        all.clear();
        for (size_t b = 0; b < beam.size(); ++b) {
            const uint64_t G = greedy_set(beam[b]);
            for (uint64_t Q : windows) {
                Child c = scan(beam[b], int(b), Q);
                if (c.ntake) all.push_back(c);
            }
            if (std::find(windows.begin(), windows.end(), G) == windows.end()) {
                Child c = scan(beam[b], int(b), G);
                if (c.ntake) all.push_back(c);
            }
        }
        if (all.empty()) return base;  // cannot happen: a gate's own qubits take it
        // a finished grouping ends the search: the cheapest one at this depth
        const Child *done = nullptr;
        for (const Child &c : all)
            if (c.ntake == beam[size_t(c.parent)].rem.size() && (!done || c.cost < done->cost)) done = &c;
        if (done) {
            std::vector<FusedGroup> out = beam[size_t(done->parent)].hist;
            out.push_back({done->Q, beam[size_t(done->parent)].rem});
            return grouping_cost(out, staged_cost) < grouping_cost(base, staged_cost) ? out : base;
        }
        std::sort(all.begin(), all.end(), [](const Child &a, const Child &b) {
            return a.score < b.score || (a.score == b.score && a.hash < b.hash);
        });
        std::vector<State> next;
        std::vector<uint64_t> seen;
        for (const Child &c : all) {
            if (int(next.size()) >= width) break;
            if (std::find(seen.begin(), seen.end(), c.hash) != seen.end()) continue;  // same gates left
            seen.push_back(c.hash);
            const State &par = beam[size_t(c.parent)];
            State st;
            st.cost = c.cost;
            st.hist = par.hist;
            FusedGroup grp{c.Q, {}};
            materialise(par, c.Q, grp.take, st.rem);
            st.hist.push_back(std::move(grp));
            next.push_back(std::move(st));
        }
        beam.swap(next);
    }
    return base;
}

std::vector<FusedGroup> fused_groups_beam(const std::vector<Gate> &gates, int k, int M, int width,
                                          double staged_cost) {
    const std::vector<FusedGroup> base = fused_groups(gates, k, M);
    const double weights[6] = {1.0, staged_cost, 0.5 * (1.0 + staged_cost), 1.15, 1.25, 1.5};
    std::vector<FusedGroup> found[6];
    run_parallel(6, [&](size_t i) { found[i] = beam_search(gates, k, M, width, weights[i], base); });
    size_t best = 0;
    for (size_t i = 1; i < 6; ++i)
        if (grouping_cost(found[i], staged_cost) < grouping_cost(found[best], staged_cost)) best = i;
    return grouping_cost(found[best], staged_cost) < grouping_cost(base, staged_cost) ? found[best] : base;
}

// Beam width of the fused grouping: the search pays off when a block pass
// is long (2^28 amplitudes and more: a block saved is ~0.3 ms or more).
constexpr int kBeamMinBits = 28;
constexpr int kBeamWidth = 8;
constexpr double kStagedCost = 1.30;  // staged / direct time of a block (measured 4.66 vs 6.04 TB/s, dense state)

void plan_fused(qsim_plan *p, int k, std::vector<__half> &rimg, double staged_cost = kStagedCost) {
    const int M = p->M;
    const size_t per = fused_rimg_halves(k);
    const std::vector<FusedGroup> groups = M >= kBeamMinBits
                                               ? fused_groups_beam(p->gates, k, M, kBeamWidth, staged_cost)
                                               : fused_groups(p->gates, k, M);
    {
        int staged = 0;
        for (const FusedGroup &g : groups) staged += (g.Q & 3u) ? 1 : 0;
        char line[160];
        std::snprintf(line, sizeof line, "grouping: %s (width %d), %zu blocks (%d holding qubit 0 or 1, staged cost %.2f)",
                      M >= kBeamMinBits ? "beam search" : "windows and greedy", M >= kBeamMinBits ? kBeamWidth : 1,
                      groups.size(), staged, staged_cost);
        p->group_log = line;
    }
    // the blocks' descriptors not yet known to the process, computed in parallel
    {
        std::vector<std::vector<int>> missing;
        std::vector<uint64_t> seen;
        for (const FusedGroup &grp : groups) {
            std::vector<int> bq;
            for (int q = 0; q < M; ++q)
                if (grp.Q & bit(q)) bq.push_back(q);
            FusedDesc d;
            if (std::find(seen.begin(), seen.end(), grp.Q) != seen.end() || desc_lookup(M, k, bq.data(), &d)) continue;
            seen.push_back(grp.Q);
            missing.push_back(bq);
        }
        const size_t nt = std::min<size_t>(missing.size(), 8);
        run_parallel(nt, [&](size_t t) {
            for (size_t i = t; i < missing.size(); i += nt) fused_desc(M, k, missing[i].data());
        });
    }
    for (const FusedGroup &grp : groups) {
        const uint64_t Q = grp.Q;
        const std::vector<int> &take = grp.take;
        int bq[8], nb = 0;
        for (int q = 0; q < M; ++q)
            if (Q & bit(q)) bq[nb++] = q;
        Step st{};
        st.type = S_FUSED;
        st.f = fused_desc(M, k, bq);
        st.rimg = rimg.size();
        rimg.resize(rimg.size() + per, __float2half_rn(0.f));
        const std::vector<double> U = block_matrix(p->gates, take, bq, k);
        st.f.unitary = is_unitary(U, k) ? 1 : 0;
        block_rimg(U, k, rimg.data() + st.rimg);
        st.bytes = 2.0 * std::ldexp(1.0, M) * 8.0;
        p->steps.push_back(st);
    }
}

// ------------------------------------------------------------ AUTO mode
// A time model for choosing the execution form (complex64): a pass or a
// block moves 16 * 2^M bytes; a register pass also spends the arithmetic of
// its ops; a permutation pass and a fused block of width k run at their own
// bandwidths.  The rates are measured on the device (tune.cu: a light and a
// heavy tile pass, a permutation pass, one fused block of each width on and
// off qubits 0..4) and kept in the tuning cache.

// Seconds of the fused blocks of width k for these gates (the grouping of
// plan_fused, without building the matrices).
double model_fused(const std::vector<Gate> &gates, int k, int M, const ModelRates &r, int *nblocks) {
    const double bytes = 16.0 * std::ldexp(1.0, M);
    double t = 0;
    const std::vector<FusedGroup> groups = fused_groups(gates, k, M);
    for (const FusedGroup &grp : groups) t += bytes / ((grp.Q & 3u) ? r.fused_staged[k] : r.fused_direct[k]);
    if (nblocks) *nblocks = int(groups.size());
    return t;
}

// FMA-equivalent operations per amplitude of one register op.
double regop_cost(const RegOp &op, int S) {
    const double touched = double(__builtin_popcount(op.smask)) / double(S) / double(1u << __builtin_popcount(op.nmask));
    const int c = op.code;
    if (c >= RC_NHAD) return 6.0;
    if (c >= RC_HAD) return 2.0;
    if (c < RC_RDENSE) return 16.0 * touched * 2.0;  // pair kinds: smask counts pairs
    if (c < RC_SWAP) return 8.0 * touched * 2.0;
    if (c < RC_PHASE_ALL) return 0.5;
    if (c == RC_TAB) return 6.0 * touched;
    if (c == RC_PHRUN) return 24.0;
    return 8.0 * touched;
}

double step_fma(const Step &st, const std::vector<RegOp> &regops) {
    if (st.type != S_TILE) return 0.0;
    double fma = 0;
    const int S = 1 << std::max(0, st.d.b - kRegThreadBits);
    if (st.d.round_count > 0)
        for (int j = 0; j < st.d.op_count; ++j) fma += regop_cost(regops[size_t(st.d.op_begin + j)], S);
    else
        fma = 16.0 * double(st.d.op_count);
    return fma;
}

}  // namespace

double qs::plan_model_fma(const qsim_plan *p) {
    double f = 0;
    for (const Step &st : p->steps) f += step_fma(st, p->h_regops);
    return f;
}

namespace {

double model_seconds(const qsim_plan *p, const std::vector<RegOp> &regops, const ModelRates &r) {
    const double N = std::ldexp(1.0, p->M);
    double t = 0;
    for (const Step &st : p->steps) {
        if (st.type == S_PERM) t += 16.0 * N / r.perm_bw;
        else if (st.type == S_TILE) t += std::max(16.0 * N / r.pass_bw, step_fma(st, regops) * N / r.fma_rate);
        else if (st.type == S_FUSED) t += 16.0 * N / r.fused_direct[st.f.k];
    }
    return t;
}

int dev_alloc(const qsim_plan *p, void **dev, size_t bytes) {
    return dmalloc(p->alloc, dev, bytes, p->alloc_stream, "plan tables");
}

void dev_free(const qsim_plan *p, void *dev, size_t bytes) { dfree(p->alloc, dev, bytes, p->alloc_stream); }

int upload(const qsim_plan *p, void **dev, const void *host, size_t bytes, size_t *out_bytes) {
    *out_bytes = bytes;
    if (bytes == 0) return QSIM_OK;
    if (int rc = dev_alloc(p, dev, bytes)) return rc;
    // pageable source: the copy has left `host` when the call returns
    if (p->alloc_stream)
        QS_CUDA(cudaMemcpyAsync(*dev, host, bytes, cudaMemcpyHostToDevice, p->alloc_stream));
    else
        QS_CUDA(cudaMemcpy(*dev, host, bytes, cudaMemcpyHostToDevice));
    return QSIM_OK;
}

int run_steps(const qsim_plan *p, void *dst, const void *src, cudaStream_t s, bool timed) {
    const size_t vec_bytes = (size_t(1) << p->M) * amp_bytes(p->prec);
    bool first = true;
    if (timed) {
        if (int rc = next_event(p, s)) return rc;
        ++p->timed_execs;
    }
    // reading a separate source, the first tile pass can apply the front
    // permutation itself: the permutation pass is skipped
    const bool absorb = p->jit_gather_k && src != dst && p->steps.size() > 1 && p->steps[0].type == S_PERM;
    p->last_absorbed = absorb;
    for (const Step &st : p->steps) {
        const size_t si = size_t(&st - p->steps.data());
        if (timed && si > 0)
            if (int rc = next_event(p, s)) return rc;
        if (absorb && si == 0) continue;
        if (absorb && si == 1) {
            if (int rc = launch_jit_pass(p->jit_gather_k, dst, src, p->M, st.d, p->d_runs, s)) return rc;
        } else if (st.type == S_TILE && st.d.round_count > 0) {
            if (si < p->jit_k.size() && p->jit_k[si]) {
                if (int rc = launch_jit_pass(p->jit_k[si], dst, first ? src : dst, p->M, st.d, p->d_runs, s)) return rc;
            } else if (int rc = launch_tile_reg(dst, first ? src : dst, p->M, st.d, p->d_regops, p->d_rounds,
                                                p->d_runs, s)) {
                return rc;
            }
        } else if (st.type == S_TILE) {
            if (int rc = launch_tile_pass(dst, first ? src : dst, p->M, p->prec, st.d, p->d_ops, p->d_runs, s))
                return rc;
        } else if (st.type == S_PERM) {
            if (int rc = launch_perm(dst, first ? src : dst, p->M, p->prec, st.perm, s)) return rc;
        } else if (st.type == S_FUSED) {
            if (int rc = launch_fused(dst, first ? src : dst, p->M, st.f, static_cast<const __half *>(p->d_rimg) + st.rimg,
                                      p->d_status, s, uint64_t(p->opts.wait_us) * 1000u))
                return rc;
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

namespace qs {

bool build_register_rounds(const std::vector<TileOp<float2>> &ops, int op_begin, int op_count, TilePassDesc &d,
                           int RB, std::vector<RegOp> &regops, std::vector<RoundDesc> &rounds,
                           std::vector<unsigned char> &runs) {
    return build_rounds(ops, op_begin, op_count, d, RB, regops, rounds, runs);
}

int smem_wavefronts(const uint32_t *addr, int width) { return wavefronts(addr, width); }

}  // namespace qs

namespace qs {

// ------------------------------------------------ touched-qubit subspace
// Section 3.2 (Figure 7) allocates the state values of a qubit only once a
// gate first uses it: every amplitude whose untouched qubits are not all 0
// is zero, and a transformation on zero values changes nothing (EQ 6 sums
// the cost of each step over the qubits used so far).  Here a circuit applied
// to |0...0> is planned the same way on a flat vector.  Qubits are numbered
// in the order a gate first touches them (virtual position v = the v-th
// qubit touched), so the nonzero amplitudes are the first 2^|T| of the
// vector, T the touched set, and gates act on that prefix only:
//   - a gate with a control outside T is the identity (the control is 0);
//   - a gate on a target outside T with U10 = 0 leaves the target at 0 and
//     multiplies the amplitudes whose controls are 1 by U00: it becomes
//     diag(1, U00) on a control (controlled by the other), or, with no
//     control, the factor U00 on the whole prefix (kept aside while T is
//     empty and folded into the first gate that touches a qubit);
//   - any other gate on a target outside T adds the target to T, doubling
//     the prefix; its new half is zero because the vector starts at |0...0>.
// Gates between two growths form a segment, run by a child plan on the
// prefix; short segments (fewer than kSubMinGates gates, or a prefix below
// 2^kSubMinBits amplitudes) are merged into the next one, whose larger
// prefix they run on unchanged (the extra amplitudes are zero).  At the end
// a permutation plan moves virtual position v to physical qubit order[v]
// (the untouched qubits, all 0, after the touched ones in ascending order):
// a product of two involutions, each one in-place permutation pass.
constexpr int kSubMinBits = 16;
constexpr size_t kSubMinGates = 8;

// Two involutions s1, s2 with s2(s1(v)) = pi(v): on each cycle
// c_0 -> c_1 -> ... of pi, s1(c_i) = c_{-i} and s2(c_i) = c_{1-i}.
void split_involutions(const std::vector<int> &pi, std::vector<int> &s1, std::vector<int> &s2) {
    const int M = int(pi.size());
    s1.assign(M, 0);
    s2.assign(M, 0);
    std::vector<char> seen(M, 0);
    for (int v = 0; v < M; ++v) {
        if (seen[v]) continue;
        std::vector<int> cyc;
        for (int c = v; !seen[c]; c = pi[c]) {
            seen[c] = 1;
            cyc.push_back(c);
        }
        const int k = int(cyc.size());
        for (int i = 0; i < k; ++i) {
            s1[cyc[i]] = cyc[(k - i) % k];
            s2[cyc[i]] = cyc[(k + 1 - i) % k];
        }
    }
}

int plan_relabel(const qsim_plan *parent, const std::vector<int> &pi, qsim_plan **out) {
    const int M = parent->M;
    qsim_plan *r = new qsim_plan();
    r->M = M;
    r->prec = parent->prec;
    r->mode = QSIM_MODE_TILED;
    r->alloc_stream = parent->alloc_stream;
    r->alloc = parent->alloc;
    std::vector<int> s1, s2;
    split_involutions(pi, s1, s2);
    for (const std::vector<int> *s : {&s1, &s2}) {
        bool ident = true;
        for (int v = 0; v < M; ++v) ident = ident && (*s)[v] == v;
        if (ident) continue;
        Step st{};
        st.type = S_PERM;
        st.perm = perm_desc(*s, M, parent->prec);
        st.bytes = 2.0 * std::ldexp(1.0, M) * double(amp_bytes(parent->prec));
        r->steps.push_back(st);
    }
    if (int rc = dev_alloc(r, reinterpret_cast<void **>(&r->d_status), sizeof(int))) {
        plan_release(r);
        return rc;
    }
    cudaError_t e = r->alloc_stream ? cudaMemsetAsync(r->d_status, 0, sizeof(int), r->alloc_stream)
                                    : cudaMemset(r->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        plan_release(r);
        return cuda_fail(e, "relabel status word");
    }
    double bytes = 0;
    for (const Step &st : r->steps) bytes += st.bytes;
    r->stats.n_passes = r->stats.n_launches = int64_t(r->steps.size());
    r->stats.mode = QSIM_MODE_TILED;
    r->stats.algo_bytes = bytes;
    *out = r;
    return QSIM_OK;
}

qsim_gate gate_record(const double *U, int t, int nc, int c0, int c1) {
    qsim_gate g{};
    for (int k = 0; k < 8; ++k) g.U[k] = U[k];
    g.target = t;
    g.ncontrols = nc;
    g.controls[0] = c0;
    g.controls[1] = c1;
    return g;
}

int plan_subspace(qsim_plan *p) {
    const int M = p->M;
    std::vector<int> virt(M, -1);
    std::vector<int> &order = p->sub_order;
    double scale[2] = {1.0, 0.0};  // factor kept aside while nothing is touched
    std::vector<std::vector<qsim_gate>> seg(1);
    std::vector<int> segM(1, 0);
    for (const Gate &g : p->gates) {
        bool live = true;
        for (int c = 0; c < g.nc; ++c) live = live && virt[g.c[c]] >= 0;
        if (!live) {
            ++p->sub_skipped;
            continue;
        }
        const double *U = g.U;
        const int vc0 = g.nc > 0 ? virt[g.c[0]] : 0, vc1 = g.nc > 1 ? virt[g.c[1]] : 0;
        if (virt[g.t] < 0 && U[4] == 0.0 && U[5] == 0.0) {  // target stays 0: factor U00 where the controls are 1
            if (U[0] == 1.0 && U[1] == 0.0) {
                ++p->sub_skipped;
                continue;
            }
            if (g.nc == 0 && order.empty()) {
                const double re = scale[0] * U[0] - scale[1] * U[1], im = scale[0] * U[1] + scale[1] * U[0];
                scale[0] = re;
                scale[1] = im;
                continue;
            }
            const double one[2] = {1.0, 0.0};
            const double *d0 = g.nc == 0 ? U : one;
            const double D[8] = {d0[0], d0[1], 0, 0, 0, 0, U[0], U[1]};
            if (g.nc == 0) seg.back().push_back(gate_record(D, 0, 0, 0, 0));
            else seg.back().push_back(gate_record(D, vc0, g.nc - 1, vc1, 0));
            continue;
        }
        double V[8];
        for (int k = 0; k < 8; ++k) V[k] = U[k];
        if (virt[g.t] < 0) {  // the target joins the touched set: a new segment on a prefix twice as long
            if (!seg.back().empty()) {
                seg.emplace_back();
                segM.push_back(0);
            }
            virt[g.t] = int(order.size());
            order.push_back(g.t);
            if (order.size() == 1 && (scale[0] != 1.0 || scale[1] != 0.0)) {  // the first touching gate has no control
                for (int k = 0; k < 8; k += 2) {
                    V[k] = scale[0] * U[k] - scale[1] * U[k + 1];
                    V[k + 1] = scale[0] * U[k + 1] + scale[1] * U[k];
                }
                scale[0] = 1.0;
                scale[1] = 0.0;
            }
        }
        segM.back() = int(order.size());
        seg.back().push_back(gate_record(V, virt[g.t], g.nc, vc0, vc1));
    }
    if (order.empty() && (scale[0] != 1.0 || scale[1] != 0.0)) {  // nothing touched: the factor on amplitude 0
        const double D[8] = {scale[0], scale[1], 0, 0, 0, 0, scale[0], scale[1]};
        seg.back().push_back(gate_record(D, 0, 0, 0, 0));
        segM.back() = 1;
    }
    // merge short segments into the next (its prefix holds theirs)
    std::vector<std::vector<qsim_gate>> mseg;
    std::vector<int> mM;
    for (size_t i = 0; i < seg.size(); ++i) {
        if (seg[i].empty()) continue;
        if (!mseg.empty() && (mM.back() < kSubMinBits || mseg.back().size() < kSubMinGates)) {
            mseg.back().insert(mseg.back().end(), seg[i].begin(), seg[i].end());
            mM.back() = segM[i];
        } else {
            mseg.push_back(seg[i]);
            mM.push_back(segM[i]);
        }
    }
    qsim_opts co = p->opts;
    co.subspace = 0;
    for (size_t i = 0; i < mseg.size(); ++i) {
        const int Ms = std::max(1, mM[i]);
        qsim_plan *c = nullptr;
        if (int rc = plan_create_on(Ms, p->prec, mseg[i].data(), mseg[i].size(), &co, p->alloc_stream, &p->alloc, &c))
            return rc;
        p->seg_plans.push_back(c);
        p->seg_M.push_back(Ms);
        p->sub_amp_updates += double(mseg[i].size()) * std::ldexp(1.0, Ms);
    }
    std::vector<int> pi(M);
    std::vector<char> used(M, 0);
    for (size_t v = 0; v < order.size(); ++v) {
        pi[v] = order[v];
        used[order[v]] = 1;
    }
    for (int q = 0, v = int(order.size()); q < M; ++q)
        if (!used[q]) pi[v++] = q;
    bool ident = true;
    for (int v = 0; v < M; ++v) ident = ident && pi[v] == v;
    if (!ident)
        if (int rc = plan_relabel(p, pi, &p->relabel)) return rc;
    p->subspace = true;
    p->mode = p->opts.mode;
    qsim_plan_stats &s = p->stats;
    s.n_gates = int64_t(p->gates.size());
    s.mode = p->opts.mode;
    s.algo_bytes = std::ldexp(1.0, M) * double(amp_bytes(p->prec));  // the initial |0...0>
    s.n_passes = s.n_launches = 1;
    for (qsim_plan *c : p->seg_plans) {
        s.n_passes += c->stats.n_passes;
        s.n_launches += c->stats.n_launches;
        s.algo_bytes += c->stats.algo_bytes;
        s.table_bytes += c->stats.table_bytes;
    }
    if (p->relabel) {
        s.n_passes += p->relabel->stats.n_passes;
        s.n_launches += p->relabel->stats.n_launches;
        s.algo_bytes += p->relabel->stats.algo_bytes;
    }
    s.amp_updates = double(p->gates.size()) * std::ldexp(1.0, M);
    return QSIM_OK;
}

// dst := circuit(|0...0>): zero the vector, run the segments on their
// prefixes, move the qubits to their own positions.
int run_subspace(const qsim_plan *p, qsim_state *dst) {
    if (int rc = launch_zero_state(dst->amps, p->M, p->prec, dst->stream)) return rc;
    for (size_t i = 0; i < p->seg_plans.size(); ++i) {
        qsim_state pre = *dst;
        pre.M = p->seg_M[i];
        if (int rc = qsim_plan_execute(p->seg_plans[i], &pre, nullptr)) return rc;
    }
    if (p->relabel)
        if (int rc = qsim_plan_execute(p->relabel, dst, nullptr)) return rc;
    return QSIM_OK;
}

int plan_create_on(int M, qsim_prec prec, const qsim_gate *gates, size_t n, const qsim_opts *opts,
                   cudaStream_t alloc_stream, const DevAllocator *alloc, qsim_plan **out) {
    if (!out) { set_error("out is NULL"); return QSIM_EINVAL; }
    if (M < 1 || M > QSIM_MAX_QUBITS) { set_error("M = %d outside [1, %d]", M, QSIM_MAX_QUBITS); return QSIM_EINVAL; }
    if (prec != QSIM_C64 && prec != QSIM_C128) { set_error("unknown precision %d", int(prec)); return QSIM_EINVAL; }
    if (n > 0 && !gates) { set_error("gates is NULL"); return QSIM_EINVAL; }
    qsim_opts o{};
    if (opts) o = *opts;
    if (o.mode < QSIM_MODE_AUTO || o.mode > QSIM_MODE_FUSED) { set_error("unknown mode %d", o.mode); return QSIM_EINVAL; }
    if (o.wait_us < 0) { set_error("wait_us %d is negative", o.wait_us); return QSIM_EINVAL; }
    if (o.tile_bits != 0 && (o.tile_bits < 6 || o.tile_bits > tile_max_bits(prec))) {
        set_error("tile_bits %d outside [6, %d]", o.tile_bits, tile_max_bits(prec));
        return QSIM_EINVAL;
    }
    qsim_plan *p = new qsim_plan();
    p->M = M;
    p->prec = prec;
    p->opts = o;
    p->alloc_stream = alloc_stream;
    p->alloc = alloc ? *alloc : current_allocator();
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
    if (o.fuse_k != 0 && (o.fuse_k < 2 || o.fuse_k > 5)) {
        set_error("fuse_k %d outside [2, 5]", o.fuse_k);
        delete p;
        return QSIM_EINVAL;
    }
    if (o.subspace) {
        if (int rc = plan_subspace(p)) {
            plan_release(p);
            return rc;
        }
        *out = p;
        return QSIM_OK;
    }
    int mode = o.mode == QSIM_MODE_AUTO ? QSIM_MODE_TILED : o.mode;
    int auto_b = 0, auto_k = 0;
    double staged_cost = kStagedCost;  // the measured ratio where AUTO has the rates
    if (o.mode == QSIM_MODE_AUTO && prec == QSIM_C64 && M >= 20) {
        // the candidates (tile passes of 2^12 or 2^11 amplitudes, fused blocks
        // of width 5, 4 or 3, unless opts fix them) planned on the host and
        // timed by the model with the device's measured rates
        ModelRates rates{};
        std::string src;
        if (int rc = model_rates(prec, o.specialize != 0 && jit_available(), &rates, &src)) {
            plan_release(p);
            return rc;
        }
        std::string log = "auto:";
        double best = 1e300;
        char line[160];
        for (int b : {12, 11}) {
            if (o.tile_bits && b != o.tile_bits) continue;
            if (b > M) continue;
            qsim_plan scratch;
            scratch.M = M;
            scratch.prec = prec;
            scratch.gates = p->gates;
            split_row_phases(scratch.gates);
            std::vector<TileOp<float2>> ops;
            std::vector<unsigned char> runs;
            std::vector<int> all(scratch.gates.size());
            for (size_t i = 0; i < all.size(); ++i) all[i] = int(i);
            plan_tiled(&scratch, b, all, ops, runs);
            std::vector<RegOp> regops;
            std::vector<RoundDesc> rounds;
            for (Step &st : scratch.steps) {
                if (st.type != S_TILE) continue;
                const int RB = st.d.b - kRegThreadBits;
                if (RB < 3 || RB > 4) continue;
                TilePassDesc d = st.d;
                if (build_rounds(ops, st.d.op_begin, st.d.op_count, d, RB, regops, rounds, runs)) st.d = d;
            }
            const double t = model_seconds(&scratch, regops, rates);
            std::snprintf(line, sizeof line, " tiled b=%d %.3g s (%zu passes),", b, t, scratch.steps.size());
            log += line;
            if (t < best) {
                best = t;
                mode = QSIM_MODE_TILED;
                auto_b = b;
                auto_k = 0;
            }
        }
        for (int k : {5, 4, 3}) {
            if (o.fuse_k && k != std::max(3, o.fuse_k)) continue;
            int nb = 0;
            const double t = model_fused(p->gates, k, M, rates, &nb);
            std::snprintf(line, sizeof line, " fused k=%d %.3g s (%d blocks),", k, t, nb);
            log += line;
            if (t < best) {
                best = t;
                mode = QSIM_MODE_FUSED;
                auto_k = k;
                auto_b = 0;
                if (rates.fused_staged[k] > 0 && rates.fused_direct[k] > 0)
                    staged_cost = rates.fused_direct[k] / rates.fused_staged[k];
            }
        }
        std::snprintf(line, sizeof line, " chosen %s %d; rates %s", mode == QSIM_MODE_FUSED ? "fused k=" : "tiled b=",
                      mode == QSIM_MODE_FUSED ? auto_k : auto_b, src.c_str());
        log += line;
        p->auto_log = log;
    }
    // The tensor-core kernel runs 4- or 5-qubit blocks of complex64 states
    // with at least 2^(k+7) amplitudes; anything else takes the tile passes.
    const int k_eff = auto_k ? auto_k : o.fuse_k == 0 ? 5 : std::max(3, o.fuse_k);
    if (mode == QSIM_MODE_FUSED && (prec != QSIM_C64 || M < kFusedTileBits)) mode = QSIM_MODE_TILED;
    p->mode = mode;
    {
        int rc = dev_alloc(p, reinterpret_cast<void **>(&p->d_status), sizeof(int));
        if (rc == QSIM_OK) {
            cudaError_t e = alloc_stream ? cudaMemsetAsync(p->d_status, 0, sizeof(int), alloc_stream)
                                         : cudaMemset(p->d_status, 0, sizeof(int));
            if (e != cudaSuccess) rc = cuda_fail(e, "plan status word");
        }
        if (rc) {
            plan_release(p);
            return rc;
        }
    }
    const size_t ab = amp_bytes(prec);
    double bytes = 0;
    if (mode == QSIM_MODE_FUSED) {
        p->fuse_k = k_eff;
        std::vector<__half> rimg;
        plan_fused(p, k_eff, rimg, staged_cost);
        int rc = fused_prepare();
        if (rc == QSIM_OK) rc = upload(p, &p->d_rimg, rimg.data(), rimg.size() * sizeof(__half), &p->rimg_bytes);
        if (rc) {
            plan_release(p);
            return rc;
        }
    } else if (mode == QSIM_MODE_UNFUSED) {
        for (const Gate &g : p->gates) {
            Step st{};
            st.type = S_GATE;
            st.g = g;
            st.bytes = gate_bytes(g, M, ab);
            p->steps.push_back(st);
        }
    } else {
        const int b = auto_b ? auto_b : o.tile_bits ? o.tile_bits : default_tile_bits(prec);
        p->tile_bits = std::min(b, M);
        int rc = tile_prepare(prec);
        if (rc == QSIM_OK && prec == QSIM_C64) rc = tile_reg_prepare();
        if (prec == QSIM_C64) split_row_phases(p->gates);
        std::vector<unsigned char> runs;
        if (rc == QSIM_OK) {
            // gate segments between runs of swaps; each swap run is one permutation pass
            std::vector<int> run_of;
            std::vector<std::vector<int>> perms;
            find_swap_runs(p->gates, run_of, perms, M);
            // all runs as one permutation at the front, when their product allows
            uint64_t reserve = 0;
            p->front_perm = swaps_to_front(p->gates, run_of, perms, M);
            if (!p->front_perm.empty()) {
                run_of.assign(p->gates.size(), -1);
                perms.clear();
                Step st{};
                st.type = S_PERM;
                st.perm = perm_desc(p->front_perm, M, prec);
                st.bytes = 2.0 * std::ldexp(1.0, M) * double(amp_bytes(prec));
                p->steps.push_back(st);
                // the first pass's tile holds the qubits of the source's low bits
                // (so that a specialised first pass can gather the permutation;
                // general and specialised plans keep the same passes)
                if (prec == QSIM_C64)
                    for (int q = 0; q < std::min(5, M); ++q) reserve |= bit(p->front_perm[q]);
            }
            std::vector<std::vector<int>> segs(1);
            std::vector<int> perm_after;  // perm_after[s] = permutation following segment s, or -1
            for (size_t gi = 0; gi < p->gates.size(); ++gi) {
                if (run_of[gi] < 0) {
                    segs.back().push_back(int(gi));
                } else if (gi == 0 || run_of[gi - 1] != run_of[gi]) {
                    perm_after.push_back(run_of[gi]);
                    segs.emplace_back();
                }
            }
            perm_after.push_back(-1);
            auto add_perm = [&](int s_idx) {
                if (perm_after[size_t(s_idx)] < 0) return;
                Step st{};
                st.type = S_PERM;
                st.perm = perm_desc(perms[size_t(perm_after[size_t(s_idx)])], M, prec);
                st.bytes = 2.0 * std::ldexp(1.0, M) * double(amp_bytes(prec));
                p->steps.push_back(st);
            };
            if (prec == QSIM_C64) {
                std::vector<TileOp<float2>> ops;
                for (size_t si = 0; si < segs.size(); ++si) {
                    plan_tiled(p, b, segs[si], ops, runs, si == 0 ? reserve : 0);
                    add_perm(int(si));
                }
                std::vector<RegOp> regops;
                std::vector<RoundDesc> rounds;
                for (Step &st : p->steps) {  // register rounds where the tile size allows
                    if (st.type != S_TILE) continue;
                    const int RB = st.d.b - kRegThreadBits;
                    if (RB < 3 || RB > 4) continue;
                    TilePassDesc d = st.d;
                    if (build_rounds(ops, st.d.op_begin, st.d.op_count, d, RB, regops, rounds, runs)) st.d = d;
                }
                carry_pass_scales(p->steps);
                rc = upload(p, &p->d_ops, ops.data(), ops.size() * sizeof(ops[0]), &p->ops_bytes);
                if (rc == QSIM_OK) rc = upload(p, &p->d_regops, regops.data(), regops.size() * sizeof(RegOp), &p->regops_bytes);
                if (rc == QSIM_OK) rc = upload(p, &p->d_rounds, rounds.data(), rounds.size() * sizeof(RoundDesc), &p->rounds_bytes);
                if (rc == QSIM_OK && o.specialize) {  // one generated kernel per register pass
                    std::vector<const TilePassDesc *> descs;
                    std::vector<size_t> at;
                    for (size_t si = 0; si < p->steps.size(); ++si)
                        if (p->steps[si].type == S_TILE && p->steps[si].d.round_count > 0) {
                            descs.push_back(&p->steps[si].d);
                            at.push_back(si);
                        }
                    // and the first tile pass once more, gathering the front
                    // permutation, if its tile covers the source's lowest 4 bits
                    std::vector<const std::vector<int> *> gathers(descs.size(), nullptr);
                    bool gather = !p->front_perm.empty() && p->steps.size() > 1 && p->steps[1].type == S_TILE &&
                                  p->steps[1].d.round_count > 0;
                    for (int q = 0; gather && q < std::min(4, M); ++q) {
                        const TilePassDesc &d1 = p->steps[1].d;
                        const int pq = p->front_perm[q];
                        bool in = pq < d1.L;
                        for (int h = 0; h < d1.nh; ++h) in = in || d1.hpos[h] == pq;
                        gather = in;
                    }
                    if (gather) {
                        descs.push_back(&p->steps[1].d);
                        gathers.push_back(&p->front_perm);
                    }
                    std::vector<cudaKernel_t> ks;
                    if (!descs.empty() &&
                        jit_build(descs, gathers, regops, rounds, runs, &p->jit_libs, &ks, &p->jit_log) == QSIM_OK) {
                        p->jit_k.assign(p->steps.size(), nullptr);
                        for (size_t j = 0; j < at.size(); ++j) p->jit_k[at[j]] = ks[j];
                        if (gather) p->jit_gather_k = ks.back();
                    }
                }
                p->h_regops = std::move(regops);
                p->h_rounds = std::move(rounds);
            } else {
                std::vector<TileOp<double2>> ops;
                for (size_t si = 0; si < segs.size(); ++si) {
                    plan_tiled(p, b, segs[si], ops, runs);
                    add_perm(int(si));
                }
                rc = upload(p, &p->d_ops, ops.data(), ops.size() * sizeof(ops[0]), &p->ops_bytes);
            }
        }
        if (rc == QSIM_OK) rc = upload(p, &p->d_runs, runs.data(), runs.size(), &p->runs_bytes);
        if (rc) {
            plan_release(p);
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
    s.fuse_k = mode == QSIM_MODE_FUSED ? p->fuse_k : 0;
    s.n_blocks = mode == QSIM_MODE_FUSED ? int32_t(p->steps.size()) : 0;
    s.algo_bytes = bytes;
    s.amp_updates = double(n) * std::ldexp(1.0, M);
    s.table_bytes = int64_t(p->ops_bytes + p->runs_bytes + p->rimg_bytes + p->regops_bytes + p->rounds_bytes);
    *out = p;
    return QSIM_OK;
}

void plan_release(qsim_plan *p) {
    if (!p) return;
    for (qsim_plan *c : p->seg_plans) plan_release(c);
    if (p->relabel) plan_release(p->relabel);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    dev_free(p, p->d_ops, p->ops_bytes);
    dev_free(p, p->d_runs, p->runs_bytes);
    dev_free(p, p->d_rimg, p->rimg_bytes);
    jit_release(p->jit_libs);
    p->jit_libs.clear();
    dev_free(p, p->d_regops, p->regops_bytes);
    dev_free(p, p->d_rounds, p->rounds_bytes);
    dev_free(p, p->d_status, sizeof(int));
    delete p;
}

}  // namespace qs

extern "C" {

int qsim_plan_create(int M, qsim_prec prec, const qsim_gate *gates, size_t n, const qsim_opts *opts,
                     qsim_plan **out) {
    return plan_create_on(M, prec, gates, n, opts, nullptr, nullptr, out);
}

int qsim_plan_execute(const qsim_plan *p, qsim_state *dst, const qsim_state *src) {
    if (!p || !dst) { set_error("plan or state is NULL"); return QSIM_EINVAL; }
    if (!src) src = dst;
    if (dst->M != p->M || dst->prec != p->prec || src->M != p->M || src->prec != p->prec) {
        set_error("state (M=%d) does not match the plan (M=%d)", dst->M, p->M);
        return QSIM_EINVAL;
    }
    if (p->subspace) return run_subspace(p, dst);  // the input is |0...0>: src is not read
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
        const bool skipped = j == 0 && p->last_absorbed;
        if (bytes) bytes[j] = skipped ? 0.0 : p->steps[j].bytes;
        if (kind) {
            const Step &st = p->steps[j];
            const bool spec = size_t(j) < p->jit_k.size() && p->jit_k[size_t(j)];
            kind[j] = skipped ? 6 : st.type == S_TILE && st.d.round_count > 0 ? (spec ? 5 : 4) : int32_t(st.type);
        }
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

int qsim_plan_describe(const qsim_plan *p, char *buf, int64_t len, int64_t *needed) {
    if (!p) { set_error("plan is NULL"); return QSIM_EINVAL; }
    if (len > 0 && !buf) { set_error("buf is NULL"); return QSIM_EINVAL; }
    std::string out;
    char line[512];
    auto add = [&](const char *fmt, auto... args) {
        std::snprintf(line, sizeof line, fmt, args...);
        out += line;
    };
    static const char *kinds[] = {"DENSE", "RDENSE", "SWAP"};
    add("M=%d prec=%s mode=%d steps=%zu\n", p->M, p->prec == QSIM_C64 ? "c64" : "c128", p->mode, p->steps.size());
    if (p->subspace) {
        add("subspace: %zu segments, %lld gates left out (control never touched), %zu qubits touched, "
            "amp-updates %.6g of %.6g flat, relabel passes %lld\n",
            p->seg_plans.size(), (long long)p->sub_skipped, p->sub_order.size(), p->sub_amp_updates,
            p->stats.amp_updates, p->relabel ? (long long)p->relabel->steps.size() : 0LL);
        add("touch order:");
        for (int q : p->sub_order) add(" %d", q);
        add("\n");
        for (size_t i = 0; i < p->seg_plans.size(); ++i) {
            const qsim_plan *c = p->seg_plans[i];
            add("segment %zu M=%d gates=%lld mode=%d passes=%lld\n", i, p->seg_M[i], (long long)c->stats.n_gates,
                c->stats.mode, (long long)c->stats.n_passes);
        }
    }
    if (!p->jit_log.empty()) add("specialisation: %s\n", p->jit_log.c_str());
    if (!p->auto_log.empty()) add("%s\n", p->auto_log.c_str());
    if (!p->group_log.empty()) add("%s\n", p->group_log.c_str());
    for (size_t j = 0; j < p->steps.size(); ++j) {
        const Step &st = p->steps[j];
        if (st.type == S_GATE) {
            add("step %zu GATE t=%d nc=%d kind=%d\n", j, st.g.t, st.g.nc, int(st.g.kind));
        } else if (st.type == S_PERM) {
            add("step %zu PERM tile_qubits=%d low=%d%s\n", j, st.perm.ns, st.perm.lb,
                j == 0 && !p->front_perm.empty()
                    ? (p->jit_gather_k ? " (swap runs moved to the front; gathered by step 1 when src != dst)"
                                       : " (swap runs moved to the front)")
                    : "");
        } else if (st.type == S_FUSED) {
            add("step %zu FUSED k=%d unitary=%d runbits=%d qubits=", j, st.f.k, st.f.unitary, st.f.runbits);
            for (int a = 0; a < st.f.k; ++a) {  // tile index bit -> device qubit
                const int b = __builtin_ctz(st.f.posA[1 << a]);
                add("%d ", b < st.f.runbits ? b : st.f.rpos[b - st.f.runbits]);
            }
            add("\n");
        } else {
            add("step %zu TILE b=%d L=%d high=", j, st.d.b, st.d.L);
            for (int h = 0; h < st.d.nh; ++h) add("%d%s", st.d.hpos[h], h + 1 < st.d.nh ? "," : "");
            const bool spec = j < p->jit_k.size() && p->jit_k[j];
            add(" ops=%d rounds=%d%s%s\n", st.d.op_count, st.d.round_count, st.d.pscale_on ? " deferred-scale" : "",
                spec ? " specialised" : "");
            for (int r = 0; r < st.d.round_count; ++r) {
                const RoundDesc &rd = p->h_rounds[size_t(st.d.round_begin + r)];
                const int RB = st.d.b - kRegThreadBits;
                add("  round %d slots=", r);
                for (int k = 0; k < RB; ++k) add("%d%s", rd.pos[k], k + 1 < RB ? "," : "");
                add(" ops:");
                for (int k = 0; k < rd.op_count; ++k) {
                    const RegOp &op = p->h_regops[size_t(st.d.op_begin + rd.op_begin + k)];
                    const int c = op.code;
                    if (c >= RC_NHAD) add(" NHAD/%d", c - RC_NHAD);
                    else if (c >= RC_HAD) add(" HAD/%d", c - RC_HAD);
                    else if (c < RC_PHASE_ALL) add(" %s%s/%d", kinds[c / 8], (c & 4) ? "p" : "", c & 3);
                    else if (c == RC_PHASE_ALL || c == RC_PHASE) add(" PHASE");
                    else if (c == RC_DIAG) add(" DIAG");
                    else if (c == RC_SCALE) add(" SCALE");
                    else if (c == RC_TAB) add(" TAB%d", op.tw);
                    else add(" PHRUN");
                    if (op.gmask) add("g");
                }
                add("\n");
            }
        }
    }
    if (needed) *needed = int64_t(out.size()) + 1;
    if (len > 0) {
        const size_t n = std::min(out.size(), size_t(len - 1));
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
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
    plan_release(p);
}

int qsim_plan_status(const qsim_plan *p) {
    if (!p) { set_error("plan is NULL"); return QSIM_EINVAL; }
    if (p->subspace) {  // the segments' plans (every record is read and cleared)
        int first = QSIM_OK;
        for (const qsim_plan *c : p->seg_plans)
            if (int rc = qsim_plan_status(c)) first = first ? first : rc;
        if (p->relabel)
            if (int rc = qsim_plan_status(p->relabel)) first = first ? first : rc;
        return first;
    }
    int v = 0;
    QS_CUDA(cudaDeviceSynchronize());
    QS_CUDA(cudaMemcpy(&v, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        QS_CUDA(cudaMemset(p->d_status, 0, sizeof(int)));
        set_error("a kernel of this plan gave up a bounded wait (status %d)", v);
        return v;
    }
    return QSIM_OK;
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
    if (rc == QSIM_OK) rc = qsim_plan_status(p);
    qsim_plan_destroy(p);
    return rc;
}

}  // extern "C"
