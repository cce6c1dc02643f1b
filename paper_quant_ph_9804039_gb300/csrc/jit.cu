// Specialised register tile passes (qsim_opts.specialize).
//
// The general register kernel (k_tile_reg.cu) reads each op's kind, slot bit,
// masks and matrix from shared memory and dispatches at run time; with a few
// floating-point operations per amplitude per gate, that dispatch is most of
// its instruction stream.  Here every register tile pass of a plan becomes its
// own kernel, generated as CUDA source at plan creation with the pass's tile
// layout, rounds, op kinds, slot masks and matrix entries as literals, and
// compiled by NVRTC for sm_103a, one program per pass on a pool of host
// threads.  The kernel also stages its tiles through shared memory with
// cp.async (the next tile in flight) and may gather a qubit permutation on
// the way in (see emit_pass).  The arithmetic is that of the general kernel
// (Section 2.1's pair update with compensated entries, unit-modulus phase
// tables, Hadamards with the factor deferred; runs of phase gates as one
// phase polynomial), op by op in the same order, so results are bitwise
// those of the general kernel.  NVRTC is loaded with
// dlopen on first use; without it, or if compilation fails, the plan keeps the
// general kernel (qsim_plan_describe says which).
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <functional>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "qsim_internal.h"

namespace qs {
namespace {

const char *const kJitHeader =
#include "jit_device_src.inc"
    ;

// ------------------------------------------------------------------ NVRTC
struct Nvrtc {
    bool tried = false, ok = false;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

Nvrtc &nvrtc() {
    static Nvrtc n;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (n.tried) return n;
    n.tried = true;
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void *h = nullptr;
    for (const char *nm : names)
        if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) return n;
    n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
    n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
    n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    n.log = reinterpret_cast<decltype(n.log)>(dlsym(h, "nvrtcGetProgramLog"));
    n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
    return n;
}

// ------------------------------------------------------------- generation
struct Src {
    std::string s;
    void operator()(const char *fmt, ...) __attribute__((format(printf, 2, 3))) {
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        std::vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        s += buf;
    }
};

std::string flit(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    char b[48];
    std::snprintf(b, sizeof b, "__int_as_float(0x%08x)", u);
    return b;
}
std::string f2lit(float2 v) { return "make_float2(" + flit(v.x) + ", " + flit(v.y) + ")"; }

// Slots of a round: bit k of slot index c <-> tile position pos[k].
uint32_t dep_of(const RoundDesc &rd, int RB, int c) {
    uint32_t o = 0;
    for (int k = 0; k < RB; ++k)
        if ((c >> k) & 1) o |= 1u << rd.pos[k];
    return o;
}

void emit_pairs(Src &out, const RegOp &op, int RB, const char *kind) {
    const int S = 1 << RB, K = op.k;
    for (int c = 0; c < S; ++c) {
        if ((c >> K) & 1) continue;
        if (!((op.smask >> c) & 1)) continue;
        const int c1 = c | (1 << K);
        if (!std::strcmp(kind, "swap")) {
            out("    { const float2 t = v[%d]; v[%d] = v[%d]; v[%d] = t; }\n", c, c, c1, c1);
        } else if (!std::strcmp(kind, "nhad")) {
            const std::string e0 = flit(op.u[0].x), e1 = flit(op.u[1].x), e2 = flit(op.u[2].x), e3 = flit(op.u[3].x);
            out("    { const float2 a = v[%d], b = v[%d]; "
                "v[%d] = make_float2(fmaf(%s, a.x, fmaf(%s, b.x, a.x + b.x)), fmaf(%s, a.y, fmaf(%s, b.y, a.y + b.y))); "
                "v[%d] = make_float2(fmaf(%s, a.x, fmaf(%s, b.x, a.x - b.x)), fmaf(%s, a.y, fmaf(%s, b.y, a.y - b.y))); }\n",
                c, c1, c, e0.c_str(), e1.c_str(), e0.c_str(), e1.c_str(), c1, e2.c_str(), e3.c_str(), e2.c_str(),
                e3.c_str());
        } else if (!std::strcmp(kind, "had")) {
            out("    { const float2 a = v[%d], b = v[%d]; v[%d] = make_float2(a.x + b.x, a.y + b.y); "
                "v[%d] = make_float2(a.x - b.x, a.y - b.y); }\n",
                c, c1, c, c1);
        } else if (!std::strcmp(kind, "real")) {
            out("    { const float2 a = v[%d], b = v[%d]; v[%d] = qs_rmad2x(%s, %s, a, %s, %s, b); "
                "v[%d] = qs_rmad2x(%s, %s, a, %s, %s, b); }\n",
                c, c1, c, flit(op.u[0].x).c_str(), flit(op.ul[0].x).c_str(), flit(op.u[1].x).c_str(),
                flit(op.ul[1].x).c_str(), c1, flit(op.u[2].x).c_str(), flit(op.ul[2].x).c_str(),
                flit(op.u[3].x).c_str(), flit(op.ul[3].x).c_str());
        } else {
            out("    { const float2 a = v[%d], b = v[%d]; v[%d] = qs_cmad2x(U0, L0, a, U1, L1, b); "
                "v[%d] = qs_cmad2x(U2, L2, a, U3, L3, b); }\n",
                c, c1, c, c1);
        }
    }
}

// Matrix entry k of an op: a literal, or (J >= 0) entry k of the J-th matrix
// held in shared memory (mu: hi parts, ml: lo parts).
std::string ment(const RegOp &op, int J, int k, bool lo) {
    if (J < 0) return f2lit(lo ? op.ul[k] : op.u[k]);
    char b[48];
    std::snprintf(b, sizeof b, "%s[%d][%d]", lo ? "ml" : "mu", J, k);
    return b;
}

void emit_op(Src &out, const RegOp &op, const RoundDesc &rd, int RB, const TilePassDesc &d,
             const std::vector<unsigned char> &runs, int J = -1) {
    const int S = 1 << RB;
    const int code = op.code;
    if (code == RC_PHRUN) {
        PhaseRunHdr h;
        std::memcpy(&h, runs.data() + op.gsel, sizeof h);
        out("  {  // phase run\n");
        out("    const unsigned char *rec = runs + %llu;\n", (unsigned long long)op.gsel);
        out("    const int buf = nrun & 1; ++nrun;\n");
        out("    qs_phrun_setup<%d, %d>(rec, tile, kTq, kOpos, ps_cl[buf], ps_ktw[buf]);\n", d.b, d.nout);
        out("    const qs_u32 *Q = reinterpret_cast<const qs_u32 *>(rec + %u);\n", h.q_offset);
        out("    const qs_u32 q0 = __ldg(Q + i0);\n");
        out("    qs_u32 phi = __ldg(reinterpret_cast<const qs_u32 *>(rec + sizeof(QsPhaseRunHdr))) + q0;\n");
        out("    #pragma unroll\n    for (int j = 0; j < 8; ++j) phi += ps_ktw[buf][j];\n");
        out("    #pragma unroll\n    for (int t = 0; t < %d; ++t) if ((i0 >> t) & 1u) phi += ps_cl[buf][t];\n", d.b);
        out("    float2 e[%d];\n    e[0] = qs_expi(phi);\n", S);
        for (int k = 0; k < RB; ++k) {
            out("    { const float2 dk = qs_expi(ps_cl[buf][%d] + __ldg(Q + (i0 | %uu)) - q0);\n", rd.pos[k],
                1u << rd.pos[k]);
            for (int c = 0; c < (1 << k); ++c) out("      e[%d] = qs_cmul(e[%d], dk);\n", c | (1 << k), c);
            out("    }\n");
        }
        out("    const float2 *f = reinterpret_cast<const float2 *>(runs + %u);\n", op.tab_off);
        for (int c = 0; c < S; ++c) out("    v[%d] = qs_cmul(qs_cmul(e[%d], __ldg(f + %d)), v[%d]);\n", c, c, c, c);
        out("  }\n");
        return;
    }
    out("  {\n");
    if (op.gmask) out("   if ((base & %lluull) == %lluull)\n", (unsigned long long)op.gmask, (unsigned long long)op.gmask);
    if (op.nmask) out("   if ((i0 & %uu) == %uu)\n", op.nmask, op.nmask);
    out("   {\n");
    if (code >= RC_NHAD) {
        emit_pairs(out, op, RB, "nhad");
    } else if (code >= RC_HAD) {
        emit_pairs(out, op, RB, "had");
    } else if (code < RC_PHASE_ALL) {
        const int fam = code / 8;  // 0 dense, 1 real, 2 swap
        if (fam == 0)
            for (int j = 0; j < 4; ++j)
                out("    const float2 U%d = %s, L%d = %s;\n", j, ment(op, J, j, false).c_str(), j, ment(op, J, j, true).c_str());
        emit_pairs(out, op, RB, fam == 0 ? "dense" : (fam == 1 ? "real" : "swap"));
    } else if (code == RC_PHASE_ALL || code == RC_PHASE) {
        out("    const float2 U3 = %s, L3 = %s;\n", ment(op, J, 3, false).c_str(), ment(op, J, 3, true).c_str());
        for (int c = 0; c < S; ++c)
            if ((op.smask >> c) & 1) out("    v[%d] = qs_cmulx(U3, L3, v[%d]);\n", c, c);
    } else if (code == RC_DIAG) {
        out("    const float2 U0 = %s, L0 = %s, U3 = %s, L3 = %s;\n", ment(op, J, 0, false).c_str(),
            ment(op, J, 0, true).c_str(), ment(op, J, 3, false).c_str(), ment(op, J, 3, true).c_str());
        if (op.tbn) out("    const bool up = (i0 & %uu) != 0;\n", op.tbn);
        for (int c = 0; c < S; ++c) {
            if (!((op.smask >> c) & 1)) continue;
            if (op.tbn)
                out("    v[%d] = up ? qs_cmulx(U3, L3, v[%d]) : qs_cmulx(U0, L0, v[%d]);\n", c, c, c);
            else if ((op.tsel >> c) & 1)
                out("    v[%d] = qs_cmulx(U3, L3, v[%d]);\n", c, c);
            else
                out("    v[%d] = qs_cmulx(U0, L0, v[%d]);\n", c, c);
        }
    } else if (code == RC_SCALE) {
        out("    const bool up = (base & %lluull) != 0;\n", (unsigned long long)op.gsel);
        out("    const float2 F = up ? %s : %s, FL = up ? %s : %s;\n", ment(op, J, 3, false).c_str(),
            ment(op, J, 0, false).c_str(), ment(op, J, 3, true).c_str(), ment(op, J, 0, true).c_str());
        for (int c = 0; c < S; ++c)
            if ((op.smask >> c) & 1) out("    v[%d] = qs_cmulx(F, FL, v[%d]);\n", c, c);
    } else if (code == RC_TAB) {
        out("    const float4 *tab = reinterpret_cast<const float4 *>(runs + %u);\n", op.tab_off);
        out("    const qs_u32 g = 0u");
        for (int j = 0; j < op.tw; ++j) out(" | (((i0 >> %d) & 1u) << %d)", op.tpos[j], j);
        out(";\n");
        for (int c = 0; c < S; ++c) {
            if (!((op.smask >> c) & 1)) continue;
            out("    { const float4 t = __ldg(tab + (g | %uu)); v[%d] = qs_cmul(make_float2(t.x, t.y), v[%d]); }\n",
                unsigned(op.cidx[c]), c, c);
        }
    }
    out("   }\n  }\n");
}

// Thread tid's base index in a round: tid with a zero inserted at each slot position.
uint32_t round_base(const RoundDesc &rd, int RB, uint32_t tid) {
    uint32_t i0 = tid;
    for (int k = 0; k < RB; ++k) {
        const int q = rd.pos[k];
        i0 = ((i0 >> q) << (q + 1)) | (i0 & ((1u << q) - 1));
    }
    return i0;
}

// Layout of a staged tile in shared memory: the index XOR up to two shifted
// copies of its higher bits, so a linear map (pos(x ^ y) = pos(x) ^ pos(y))
// and a bijection (each term moves bits to lower positions only).
// keep0: the tile arrives as 16-byte chunks (amplitudes 2j, 2j + 1) and the
// terms act on the chunk index j; with shifts >= 3 the 8 consecutive chunks
// that a quarter-warp copies stay on distinct banks.  Otherwise (8-byte
// copies, the gathering first pass) they act on the amplitude index.  Shifts
// and masks are chosen per pass with the bank model over the first round's
// reads (16-byte reads of both slots' amplitudes when a slot is on tile
// position 0 and pairs stay adjacent) and, for 8-byte copies, the writes.
struct Stage {
    int sh[2] = {3, 3};
    uint32_t mask[2] = {0, 0};
    bool keep0 = true;
    uint32_t pos(uint32_t x) const {
        const int k = keep0 ? 1 : 0;
        uint32_t f = 0;
        for (int t = 0; t < 2; ++t) f ^= ((x >> (sh[t] + k)) & mask[t]) << k;
        return x ^ f;
    }
};

// A gathering first pass: element u of the source-order enumeration of a
// tile (u's bit k <-> source bit sbit[k]) is tile-local index scatter(u)
// (u's bit k <-> tile position lam[k]).
struct Gather {
    int lam[32];
    int sbit[32];
    uint32_t scatter(uint32_t u, int b) const {
        uint32_t x = 0;
        for (int k = 0; k < b; ++k)
            if ((u >> k) & 1) x |= 1u << lam[k];
        return x;
    }
};

Stage choose_stage(const TilePassDesc &d, const RoundDesc &rd, int RB, const Gather *ga) {
    const int S = 1 << RB;
    auto cost = [&](const Stage &g) {
        const bool pair = rd.pos[0] == 0 && g.keep0;
        long c = 0;
        uint32_t addr[32];
        for (uint32_t w = 0; w < 8; ++w)
            for (int r = 0; r < S; r += pair ? 2 : 1) {
                for (uint32_t l = 0; l < 32; ++l) addr[l] = 8u * g.pos(round_base(rd, RB, 32 * w + l) | dep_of(rd, RB, r));
                c += smem_wavefronts(addr, pair ? 16 : 8);
            }
        if (ga)  // the copies' writes, 8 bytes per lane
            for (uint32_t u0 = 0; u0 < (1u << d.b); u0 += 32) {
                for (uint32_t l = 0; l < 32; ++l) addr[l] = 8u * g.pos(ga->scatter(u0 + l, d.b));
                c += smem_wavefronts(addr, 8);
            }
        return c;
    };
    Stage best;
    best.keep0 = ga == nullptr;
    long best_cost = cost(best);
    const uint32_t masks[] = {7u, 15u, 31u};
    auto consider = [&](const Stage &g) {
        const long c = cost(g);
        if (c < best_cost) {
            best_cost = c;
            best = g;
        }
    };
    if (!ga) {  // 16-byte chunks: one term
        for (int sh = 3; sh <= d.b - 2; ++sh)
            for (uint32_t m : masks) {
                Stage g;
                g.sh[0] = sh;
                g.mask[0] = m;
                consider(g);
            }
        return best;
    }
    for (int sh = 1; sh <= d.b - 1; ++sh)  // 8-byte copies: one or two terms
        for (uint32_t m : masks) {
            Stage g;
            g.keep0 = false;
            g.sh[0] = sh;
            g.mask[0] = m;
            consider(g);
            for (int sh2 = sh + 1; sh2 <= d.b - 1; ++sh2)
                for (uint32_t m2 : masks) {
                    g.sh[1] = sh2;
                    g.mask[1] = m2;
                    consider(g);
                }
        }
    return best;
}

// One pass as a kernel.  Each block walks its tiles with the next tile's
// amplitudes in flight (cp.async into the second of two shared-memory
// buffers) while the current one goes through the register rounds; the first
// round reads the staged tile, later rounds exchange through the same buffer,
// and the last round stores straight to device memory.  A leading op-free
// round (kept by the general kernel to read device memory coalesced) is
// skipped: the staged copy is coalesced whatever the first round's slots.
//
// With `gather` (a qubit permutation, an involution) the pass also applies
// that permutation to its input on the way in: the amplitude of physical
// index y is read from source index x, bit gather[q] of x = bit q of y.  Its
// tile holds the qubits whose source bits are 0..3 or more, so each warp
// still reads whole runs of the source; the copies are 8 bytes each, in
// source order, into the shared-memory layout chosen for them.
std::string emit_pass(int idx, const TilePassDesc &d, const std::vector<RegOp> &regops,
                      const std::vector<RoundDesc> &rounds, const std::vector<unsigned char> &runs,
                      const std::vector<int> *gather = nullptr) {
    const int RB = d.b - kRegThreadBits, S = 1 << RB;
    Src out;
    int tq[32];
    for (int t = 0; t < d.b; ++t) tq[t] = t < d.L ? t : d.hpos[t - d.L];
    const uint32_t lowmask = (1u << d.L) - 1;
    auto goff_const = [&](uint32_t i) {  // device offset of tile-local index i
        uint64_t o = i & lowmask;
        for (int h = 0; h < d.nh; ++h)
            if ((i >> (d.L + h)) & 1) o |= uint64_t(1) << d.hpos[h];
        return o;
    };
    auto swz = [](uint32_t x) { return x ^ ((x >> 4) & 15u); };
    const int r0 = d.round_count > 1 && rounds[size_t(d.round_begin)].op_count == 0 ? 1 : 0;
    const RoundDesc &rd0 = rounds[size_t(d.round_begin + r0)];
    Gather ga{};
    if (gather) {  // tile positions in the order of their source bits
        int order[32];
        for (int t = 0; t < d.b; ++t) order[t] = t;
        std::sort(order, order + d.b, [&](int a, int c) { return (*gather)[tq[a]] < (*gather)[tq[c]]; });
        for (int k = 0; k < d.b; ++k) {
            ga.lam[k] = order[k];
            ga.sbit[k] = (*gather)[tq[order[k]]];
        }
    }
    const Stage stg = choose_stage(d, rd0, RB, gather ? &ga : nullptr);
    const bool pair0 = rd0.pos[0] == 0 && stg.keep0;
    const int nchunk = 1 << (d.b - 1 - kRegThreadBits);  // 16-byte chunks per thread and tile
    auto emit_pos = [&](const char *name, const char *x) {  // name = stg.pos(x)
        const int k = stg.keep0 ? 1 : 0;
        out("  const qs_u32 %s = %s", name, x);
        for (int t = 0; t < 2; ++t)
            if (stg.mask[t]) out(" ^ (((%s >> %d) & %uu) << %d)", x, stg.sh[t] + k, stg.mask[t], k);
        out(";\n");
    };

    out("__constant__ int kTq_%d[%d] = {", idx, d.b);
    for (int t = 0; t < d.b; ++t) out("%d%s", tq[t], t + 1 < d.b ? ", " : "};\n");
    out("__constant__ int kOpos_%d[%d] = {", idx, d.nout > 0 ? d.nout : 1);
    if (d.nout == 0) out("0};\n");
    for (int k = 0; k < d.nout; ++k) out("%d%s", d.opos[k], k + 1 < d.nout ? ", " : "};\n");
    out("extern \"C\" __global__ void __launch_bounds__(256, 3)\n");
    out("qs_pass_%d(float2 *dst, const float2 *src, const unsigned char *__restrict__ runs, qs_u64 ntiles) {\n", idx);
    out("  const int *kTq = kTq_%d; const int *kOpos = kOpos_%d; (void)kTq; (void)kOpos;\n", idx, idx);
    out("  extern __shared__ __align__(16) float2 qs_sm[];\n");
    out("  __shared__ qs_u32 ps_cl[2][16], ps_ktw[2][8];\n  int nrun = 0; (void)nrun;\n");
    out("  const qs_u32 tid = threadIdx.x;\n  float2 v[%d];\n", S);
    auto emit_base = [&](const char *name, const char *tile, bool src_bits) {
        out("   const qs_u64 %s = 0", name);
        for (int k = 0; k < d.nout; ++k)
            out(" | (((%s >> %d) & 1ull) << %d)", tile, k, src_bits ? (*gather)[d.opos[k]] : d.opos[k]);
        out(";\n");
    };
    std::function<void(const char *, const char *)> emit_issue;
    if (!gather) {
        // device offset of tile-local index 2 tid (the thread's first chunk)
        out("  const qs_u64 ld_off = (qs_u64)((tid << 1) & %uu)", lowmask);
        for (int t = std::max(1, d.L); t <= kRegThreadBits; ++t)
            out(" | ((qs_u64)((tid >> %d) & 1u) << %d)", t - 1, d.hpos[t - d.L]);
        out(";\n");
        emit_issue = [&](const char *tile, const char *buf) {
            out("   {\n");
            emit_base("nb", tile, false);
            out("   const float2 *g = src + (nb | ld_off);\n");
            out("   const qs_u32 sa = (qs_u32)__cvta_generic_to_shared(%s);\n", buf);
            for (int k = 0; k < nchunk; ++k) {
                out("   { const qs_u32 j = tid + %uu; asm volatile(\"cp.async.cg.shared.global [%%0], [%%1], 16;\" :: "
                    "\"r\"(sa + ((j ^ ((j >> %d) & %uu)) << 4)), \"l\"(g + %lluull) : \"memory\"); }\n",
                    unsigned(k << kRegThreadBits), stg.sh[0], stg.mask[0],
                    (unsigned long long)goff_const(uint32_t(k) << (kRegThreadBits + 1)));
            }
            out("   asm volatile(\"cp.async.commit_group;\" ::: \"memory\");\n   }\n");
        };
    } else {
        // element u = tid + 256 k of the source-order enumeration: its source
        // offset within the tile and (laid out) shared-memory position
        out("  const qs_u32 lx = 0u");
        for (int k = 0; k < kRegThreadBits; ++k) out(" | (((tid >> %d) & 1u) << %d)", k, ga.lam[k]);
        out(";\n");
        out("  const qs_u64 ld_off = 0ull");
        for (int k = 0; k < kRegThreadBits; ++k) out(" | ((qs_u64)((tid >> %d) & 1u) << %d)", k, ga.sbit[k]);
        out(";\n");
        emit_pos("plx", "lx");
        emit_issue = [&](const char *tile, const char *buf) {
            out("   {\n");
            emit_base("nb", tile, true);
            out("   const float2 *g = src + (nb | ld_off);\n");
            out("   const qs_u32 sa = (qs_u32)__cvta_generic_to_shared(%s);\n", buf);
            for (uint32_t k = 0; k < (1u << (d.b - kRegThreadBits)); ++k) {
                uint64_t so = 0;
                for (int j = 0; j < d.b - kRegThreadBits; ++j)
                    if ((k >> j) & 1) so |= uint64_t(1) << ga.sbit[kRegThreadBits + j];
                const uint32_t xc = ga.scatter(k << kRegThreadBits, d.b);
                out("   asm volatile(\"cp.async.ca.shared.global [%%0], [%%1], 8;\" :: \"r\"(sa + ((plx ^ %uu) << 3)), "
                    "\"l\"(g + %lluull) : \"memory\");\n",
                    stg.pos(xc), (unsigned long long)so);
            }
            out("   asm volatile(\"cp.async.commit_group;\" ::: \"memory\");\n   }\n");
        };
    }
    out("  float2 *const sb0 = qs_sm, *const sb1 = qs_sm + %u;\n", 1u << d.b);
    out("  if (blockIdx.x < ntiles) {\n   const qs_u64 t0 = blockIdx.x;\n");
    emit_issue("t0", "sb0");
    out("  }\n  qs_u32 it = 0;\n");
    out("  for (qs_u64 tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {\n");
    out("   float2 *const s = (it & 1u) ? sb1 : sb0;\n");
    out("   asm volatile(\"cp.async.wait_group 0;\" ::: \"memory\");\n   __syncthreads();\n");
    out("   if (tile + gridDim.x < ntiles) {\n   float2 *const nbuf = (it & 1u) ? sb0 : sb1;\n");
    out("   const qs_u64 nt = tile + gridDim.x;\n");
    emit_issue("nt", "nbuf");
    out("   }\n");
    emit_base("base", "tile", false);
    for (int r = r0; r < d.round_count; ++r) {
        const RoundDesc &rd = rounds[size_t(d.round_begin + r)];
        const bool last = r + 1 == d.round_count;
        out("   {  // round %d\n", r);
        out("   qs_u32 i0 = tid;\n");
        for (int k = 0; k < RB; ++k) {
            const int q = rd.pos[k];
            out("   i0 = ((i0 >> %d) << %d) | (i0 & %uu);\n", q, q + 1, (1u << q) - 1);
        }
        if (last) {
            out("   const qs_u64 gi0 = (qs_u64)(i0 & %uu)", lowmask);
            for (int h = 0; h < d.nh; ++h) out(" | ((qs_u64)((i0 >> %d) & 1u) << %d)", d.L + h, d.hpos[h]);
            out(";\n");
        }
        if (r > r0 || !last) out("   const qs_u32 si0 = i0 ^ ((i0 >> 4) & 15u);\n");
        if (r == r0) {
            emit_pos("p0", "i0");
            if (pair0) {
                out("   const float4 *s4 = reinterpret_cast<const float4 *>(s);\n");
                for (int c = 0; c < S; c += 2)
                    out("   { const float4 t = s4[(p0 ^ %uu) >> 1]; v[%d] = make_float2(t.x, t.y); "
                        "v[%d] = make_float2(t.z, t.w); }\n",
                        stg.pos(dep_of(rd, RB, c)), c, c + 1);
            } else {
                for (int c = 0; c < S; ++c) out("   v[%d] = s[p0 ^ %uu];\n", c, stg.pos(dep_of(rd, RB, c)));
            }
        } else {
            for (int c = 0; c < S; ++c) out("   v[%d] = s[si0 ^ %uu];\n", c, swz(dep_of(rd, RB, c)));
        }
        for (int k = 0; k < rd.op_count; ++k)
            emit_op(out, regops[size_t(d.op_begin + rd.op_begin + k)], rd, RB, d, runs);
        if (last) {
            if (d.pscale_on)
                for (int c = 0; c < S; ++c)
                    out("   v[%d] = make_float2(fmaf(v[%d].x, %s, v[%d].x * %s), fmaf(v[%d].y, %s, v[%d].y * %s));\n", c,
                        c, flit(d.pscale_hi).c_str(), c, flit(d.pscale_lo).c_str(), c, flit(d.pscale_hi).c_str(), c,
                        flit(d.pscale_lo).c_str());
            for (int c = 0; c < S; ++c)
                out("   dst[base | gi0 | %lluull] = v[%d];\n", (unsigned long long)goff_const(dep_of(rd, RB, c)), c);
        } else {
            out("   __syncthreads();\n");
            for (int c = 0; c < S; ++c) out("   s[si0 ^ %uu] = v[%d];\n", swz(dep_of(rd, RB, c)), c);
            out("   __syncthreads();\n");
        }
        out("   }\n");
    }
    out("  }\n}\n\n");
    return out.s;
}

// The persistent trajectory kernel (see trajectories.cu): each CTA takes
// the next trajectory from a counter and runs the circuit's passes on its
// private workspace (2^M amplitudes) in register rounds; at the start of a
// pass it builds that pass's erroneous matrices (FP64) into shared memory.
// The first pass starts from |0...0>, the last accumulates the overlap with
// the error-free state.  Op j of a pass is regops[pass op_begin + j]; its
// gate is the trajectory op src[j] (index into the plan's op table).
std::string emit_traj(int M, const std::vector<TilePassDesc> &passes, const std::vector<RegOp> &regops,
                      const std::vector<RoundDesc> &rounds, const std::vector<std::vector<int>> &src, int min_blocks,
                      int lanes) {
    Src out;
    int maxops = 1, maxb = 1;
    bool smem_tile = false;
    for (const TilePassDesc &d : passes) {
        maxops = std::max(maxops, d.op_count);
        maxb = std::max(maxb, d.b);
        smem_tile |= d.round_count > 1;
    }
    for (size_t p = 0; p < passes.size(); ++p) {
        out("__constant__ int kSrc_%zu[%d] = {", p, std::max<int>(1, int(src[p].size())));
        if (src[p].empty()) out("0");
        for (size_t j = 0; j < src[p].size(); ++j) out("%d%s", src[p][j], j + 1 < src[p].size() ? ", " : "");
        out("};\n");
    }
    // `lanes` trajectories per CTA (256 threads each) run the same code in
    // lockstep: the CTA's barriers keep them at the same place in the kernel,
    // so the instruction cache serves both (with two CTAs per SM at different
    // places in this long, fully unrolled kernel, warps stalled most on
    // instruction fetch).  Each lane has its own workspace, tile buffer,
    // matrices and sums; a lane past the last trajectory repeats its CTA's
    // first one and writes nothing.
    out("extern \"C\" __global__ void __launch_bounds__(%d, %d)\n", 256 * lanes, min_blocks);
    out("qs_traj(const QsTrajOp *__restrict__ ops, const double *__restrict__ eps, int n, int T,\n"
        "        const float2 *__restrict__ ideal, float2 *work, double *__restrict__ F_out, unsigned *counter) {\n");
    out("  const qs_u32 lane = threadIdx.x >> 8;\n");
    if (smem_tile && lanes > 1)  // dynamic: two tiles of 2^12 pass the 48 KB static limit
        out("  extern __shared__ float2 s_dyn[];\n  float2 *s = s_dyn + lane * %du;\n", 1u << maxb);
    else if (smem_tile)
        out("  __shared__ float2 s[%d];\n", 1 << maxb);
    out("  __shared__ float2 mu_all[%d][%d][4], ml_all[%d][%d][4];\n", lanes, maxops, lanes, maxops);
    out("  float2 (*mu)[4] = mu_all[lane];\n  float2 (*ml)[4] = ml_all[lane];\n");
    out("  __shared__ double red_all[%d][2][8];\n  double (*red)[8] = red_all[lane];\n  __shared__ int s_t;\n", lanes);
    out("  float2 *ws = work + ((qs_u64)(blockIdx.x * %d + lane) << %d);\n", lanes, M);
    out("  const qs_u32 tid = threadIdx.x & 255u;\n  float2 v[16];\n");
    out("  for (;;) {\n   if (threadIdx.x == 0) s_t = int(atomicAdd(counter, %du));\n   __syncthreads();\n", lanes);
    out("   const int t0 = s_t;\n   if (t0 >= T) break;\n");
    out("   const bool live = t0 + int(lane) < T;\n   const int t = live ? t0 + int(lane) : t0;\n");
    out("   double ore = 0.0, oim = 0.0;\n");
    for (size_t p = 0; p < passes.size(); ++p) {
        const TilePassDesc &d = passes[p];
        const int RB = d.b - kRegThreadBits, S = 1 << RB;
        const bool first = p == 0, last = p + 1 == passes.size();
        out("   {  // pass %zu\n", p);
        out("   __syncthreads();\n");
        out("   for (int j = tid; j < %d; j += 256) { const QsTrajOp &op = ops[kSrc_%zu[j]]; "
            "qs_noisy_matrix(op, eps[(qs_u64)t * n + op.gate], mu[j], ml[j]); }\n",
            d.op_count, p);
        out("   __syncthreads();\n");
        const uint32_t lowmask = (1u << d.L) - 1;
        auto goff_const = [&](uint32_t i) {
            uint64_t o = i & lowmask;
            for (int h = 0; h < d.nh; ++h)
                if ((i >> (d.L + h)) & 1) o |= uint64_t(1) << d.hpos[h];
            return o;
        };
        auto swz = [](uint32_t x) { return x ^ ((x >> 4) & 15u); };
        out("   for (qs_u64 tile = 0; tile < %lluull; ++tile) {\n", 1ull << d.nout);
        out("    const qs_u64 base = 0");
        for (int k = 0; k < d.nout; ++k) out(" | (((tile >> %d) & 1ull) << %d)", k, d.opos[k]);
        out(";\n");
        for (int r = 0; r < d.round_count; ++r) {
            const RoundDesc &rd = rounds[size_t(d.round_begin + r)];
            out("    {  // round %d\n    qs_u32 i0 = tid;\n", r);
            for (int k = 0; k < RB; ++k) {
                const int q = rd.pos[k];
                out("    i0 = ((i0 >> %d) << %d) | (i0 & %uu);\n", q, q + 1, (1u << q) - 1);
            }
            if (r == 0 || r + 1 == d.round_count) {
                out("    const qs_u64 gi0 = (qs_u64)(i0 & %uu)", lowmask);
                for (int h = 0; h < d.nh; ++h) out(" | ((qs_u64)((i0 >> %d) & 1u) << %d)", d.L + h, d.hpos[h]);
                out(";\n");
            }
            if (d.round_count > 1) out("    const qs_u32 si0 = i0 ^ ((i0 >> 4) & 15u);\n");
            for (int c = 0; c < S; ++c) {
                const unsigned long long gd = (unsigned long long)goff_const(dep_of(rd, RB, c));
                if (r == 0 && first)
                    out("    v[%d] = make_float2((base | gi0 | %lluull) == 0ull ? 1.f : 0.f, 0.f);\n", c, gd);
                else if (r == 0)
                    out("    v[%d] = ws[base | gi0 | %lluull];\n", c, gd);
                else
                    out("    v[%d] = s[si0 ^ %uu];\n", c, swz(dep_of(rd, RB, c)));
            }
            for (int k = 0; k < rd.op_count; ++k) {
                const int j = rd.op_begin + k;  // op index within the pass
                std::vector<unsigned char> none;
                emit_op(out, regops[size_t(d.op_begin + j)], rd, RB, d, none, j);
            }
            if (r + 1 == d.round_count) {
                for (int c = 0; c < S; ++c) {
                    const unsigned long long gd = (unsigned long long)goff_const(dep_of(rd, RB, c));
                    if (last)
                        out("    { const float2 a = ideal[base | gi0 | %lluull]; ore += (double)fmaf(a.x, v[%d].x, a.y * v[%d].y); "
                            "oim += (double)fmaf(a.x, v[%d].y, -a.y * v[%d].x); }\n",
                            gd, c, c, c, c);
                    else
                        out("    ws[base | gi0 | %lluull] = v[%d];\n", gd, c);
                }
            } else {
                out("    __syncthreads();\n");
                for (int c = 0; c < S; ++c) out("    s[si0 ^ %uu] = v[%d];\n", swz(dep_of(rd, RB, c)), c);
                out("    __syncthreads();\n");
            }
            out("    }\n");
        }
        out("   }\n   }\n");
    }
    out("   for (int o = 16; o > 0; o >>= 1) { ore += __shfl_xor_sync(0xffffffffu, ore, o); "
        "oim += __shfl_xor_sync(0xffffffffu, oim, o); }\n");
    out("   if ((tid & 31) == 0) { red[0][tid >> 5] = ore; red[1][tid >> 5] = oim; }\n   __syncthreads();\n");
    out("   if (tid == 0 && live) { double a = 0, b = 0; for (int w = 0; w < 8; ++w) { a += red[0][w]; b += red[1][w]; } "
        "F_out[t] = a * a + b * b; }\n");
    out("   __syncthreads();\n  }\n}\n");
    return out.s;
}

// Compile one program for sm_103a; false (and *log) on failure.
bool compile_cubin(const std::string &src, const char *name, std::vector<char> *cubin, std::string *log) {
    Nvrtc &n = nvrtc();
    nvrtcProgram prog;
    if (n.create(&prog, src.c_str(), name, 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        *log = "nvrtcCreateProgram failed";
        return false;
    }
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17"};
    if (n.compile(prog, 2, opts) != NVRTC_SUCCESS) {
        size_t ls = 0;
        n.log_size(prog, &ls);
        std::string l(ls, '\0');
        if (ls) n.log(prog, &l[0]);
        *log = "NVRTC compilation failed: " + l.substr(0, 2000);
        n.destroy(&prog);
        return false;
    }
    size_t cs = 0;
    n.cubin_size(prog, &cs);
    cubin->resize(cs);
    n.cubin(prog, cubin->data());
    n.destroy(&prog);
    return true;
}

}  // namespace

bool jit_available() { return nvrtc().ok; }

// One program per pass, compiled on a pool of host threads (compile time
// grows faster than linearly with the program, and passes are independent),
// each loaded as its own library.
int jit_build(const std::vector<const TilePassDesc *> &passes, const std::vector<const std::vector<int> *> &gathers,
              const std::vector<RegOp> &regops, const std::vector<RoundDesc> &rounds,
              const std::vector<unsigned char> &runs, std::vector<cudaLibrary_t> *libs,
              std::vector<cudaKernel_t> *kernels, std::string *log) {
    if (!nvrtc().ok) {
        if (log) *log = "NVRTC not found";
        return QSIM_EUNSUPPORTED;
    }
    const size_t np = passes.size();
    std::vector<std::string> srcs(np), logs(np);
    for (size_t i = 0; i < np; ++i) srcs[i] = std::string(kJitHeader) + emit_pass(0, *passes[i], regops, rounds, runs, i < gathers.size() ? gathers[i] : nullptr);
    std::vector<std::vector<char>> cubins(np);
    std::vector<char> ok(np, 0);
    std::atomic<size_t> next{0};
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (unsigned w = 0; w < std::min<unsigned>(hw, unsigned(np)); ++w)
        pool.emplace_back([&]() {
            for (size_t i; (i = next.fetch_add(1)) < np;) ok[i] = compile_cubin(srcs[i], "qsim_pass.cu", &cubins[i], &logs[i]);
        });
    for (std::thread &t : pool) t.join();
    for (size_t i = 0; i < np; ++i)
        if (!ok[i]) {
            if (log) *log = logs[i];
            return QSIM_EUNSUPPORTED;
        }
    libs->assign(np, nullptr);
    kernels->assign(np, nullptr);
    for (size_t i = 0; i < np; ++i) {
        cudaError_t e = cudaLibraryLoadData(&(*libs)[i], cubins[i].data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        if (e == cudaSuccess) e = cudaLibraryGetKernel(&(*kernels)[i], (*libs)[i], "qs_pass_0");
        int dev = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess)  // two staged tiles
            e = cudaKernelSetAttributeForDevice((*kernels)[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                int(jit_pass_smem_bytes(*passes[i])), dev);
        if (e != cudaSuccess) {
            jit_release(*libs);
            libs->clear();
            return cuda_fail(e, "loading a specialised pass");
        }
    }
    return QSIM_OK;
}

int jit_build_traj(int M, const std::vector<TilePassDesc> &passes, const std::vector<RegOp> &regops,
                   const std::vector<RoundDesc> &rounds, const std::vector<std::vector<int>> &src, int min_blocks,
                   int lanes, cudaLibrary_t *lib, cudaKernel_t *kernel, std::string *log) {
    if (!nvrtc().ok) {
        if (log) *log = "NVRTC not found";
        return QSIM_EUNSUPPORTED;
    }
    const std::string text = std::string(kJitHeader) + emit_traj(M, passes, regops, rounds, src, min_blocks, lanes);
    std::vector<char> cubin;
    std::string l;
    if (!compile_cubin(text, "qsim_traj.cu", &cubin, &l)) {
        if (log) *log = l;
        return QSIM_EUNSUPPORTED;
    }
    cudaError_t e = cudaLibraryLoadData(lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) return cuda_fail(e, "loading the trajectory kernel");
    e = cudaLibraryGetKernel(kernel, *lib, "qs_traj");
    int dev = 0;
    if (e == cudaSuccess && lanes > 1) e = cudaGetDevice(&dev);
    if (e == cudaSuccess && lanes > 1)
        e = cudaKernelSetAttributeForDevice(*kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            int(jit_traj_smem_bytes(passes, lanes)), dev);
    if (e != cudaSuccess) {
        cudaLibraryUnload(*lib);
        *lib = nullptr;
        return cuda_fail(e, "finding the trajectory kernel");
    }
    return QSIM_OK;
}

size_t jit_pass_smem_bytes(const TilePassDesc &d) { return size_t(2) * sizeof(float2) << d.b; }

size_t jit_traj_smem_bytes(const std::vector<TilePassDesc> &passes, int lanes) {
    if (lanes < 2) return 0;
    int maxb = 1;
    for (const TilePassDesc &d : passes) maxb = std::max(maxb, d.b);
    return size_t(lanes) * sizeof(float2) << maxb;
}

void jit_release(cudaLibrary_t lib) {
    if (lib) cudaLibraryUnload(lib);
}

void jit_release(const std::vector<cudaLibrary_t> &libs) {
    for (cudaLibrary_t l : libs) jit_release(l);
}

int launch_jit_pass(cudaKernel_t k, void *dst, const void *src, int M, const TilePassDesc &d, const void *runs_dev,
                    cudaStream_t s) {
    unsigned long long ntiles = 1ull << (M - d.b);
    uint64_t grid = uint64_t(num_sms()) * 3;  // __launch_bounds__(256, 3), one wave of resident blocks
    if (grid > ntiles) grid = ntiles;
    void *dp = dst;
    const void *sp = src;
    const void *rp = runs_dev;
    void *args[] = {&dp, &sp, &rp, &ntiles};
    QS_CUDA(cudaLaunchKernel(reinterpret_cast<const void *>(k), dim3(unsigned(grid)), dim3(256), args,
                             jit_pass_smem_bytes(d), s));
    return QSIM_OK;
}

}  // namespace qs
