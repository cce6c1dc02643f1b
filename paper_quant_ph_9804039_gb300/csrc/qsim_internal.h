// Internal declarations shared by the translation units of the CUDA path.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <type_traits>
#include <vector>

#include "qsim.h"

namespace qs {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);  // records the message, returns QSIM_ECUDA
#define QS_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return qs::cuda_fail(e_, #call); \
    } while (0)
#define QS_CHECK_LAUNCH(what)                           \
    do {                                                \
        cudaError_t e_ = cudaGetLastError();            \
        if (e_ != cudaSuccess) return qs::cuda_fail(e_, what); \
    } while (0)

int num_sms();  // streaming multiprocessors of the current device

// ----------------------------------------------------------- device memory
// The function pair in force when an object was created (qsim_set_allocator;
// null = the CUDA runtime).  dmalloc returns QSIM_ENOMEM (message set) on
// failure; with s != nullptr and no hook the runtime allocation is
// stream-ordered (cudaMallocAsync / cudaFreeAsync on s).
struct DevAllocator {
    qsim_device_alloc_fn alloc;
    qsim_device_free_fn free;
    void *ctx;
};
DevAllocator current_allocator();
int dmalloc(const DevAllocator &a, void **p, size_t bytes, cudaStream_t s, const char *what);
void dfree(const DevAllocator &a, void *p, size_t bytes, cudaStream_t s);

// ------------------------------------------------------------- autotuning
// Rates of the execution forms measured on the device (tune.cu), in bytes/s
// (read + write) or FMA-equivalents/s; fused rates per block width k, for
// blocks off qubits 0..4 (direct stores) and on them (staged stores).
struct ModelRates {
    double pass_bw, fma_rate, perm_bw;
    double fused_direct[6], fused_staged[6];
};
int model_rates(qsim_prec prec, bool specialised, ModelRates *r, std::string *source);
// A persisted value under `key` in the tuning cache (1 if found).
int tune_lookup(const std::string &key, double *value);
void tune_record(const std::string &key, double value);
std::string tune_device_key();
double plan_model_fma(const ::qsim_plan *p);  // FMA-equivalents per amplitude over the plan's tile passes

// ------------------------------------------------------------------- gates
// Gate kinds, chosen from the matrix on the host:
//   DENSE  : general 2x2
//   DIAG   : U01 = U10 = 0
//   PHASE1 : U01 = U10 = 0 and U00 = 1 exactly (only target-1 states change)
//   SWAPX  : U = X exactly (a pure exchange, no arithmetic)
//   SCALE  : (tile passes only) a diagonal gate whose target lies outside the
//            tile: one factor per tile, U00 or U11 chosen by the tile's index.
//   PHRUN  : (tile passes only) a run of diagonal gates with unit-modulus
//            entries and at most one control, applied at once as a phase
//            polynomial of the index bits (see PhaseRun).
//   TAB    : (register rounds) a run of phase gates inside the tile, one
//            table lookup per amplitude.
//   RDENSE : (register rounds) a dense gate with real entries.
enum Kind : uint32_t {
    K_DENSE = 0, K_DIAG = 1, K_PHASE1 = 2, K_SWAPX = 3, K_SCALE = 4, K_PHRUN = 5, K_TAB = 6, K_RDENSE = 7
};

struct Gate {
    double U[8];
    int t;
    int nc;
    int c[2];
    uint64_t cmask;  // all control bits
    Kind kind;
    bool nondiag() const { return kind == K_DENSE || kind == K_SWAPX; }
};

// Validate a record and classify its matrix.  Returns QSIM_OK or QSIM_EINVAL.
int make_gate(int M, const double *U, int target, const int *controls, int ncontrols, Gate *out);

// Algorithmic bytes (read + write) of one gate applied on its own.
double gate_bytes(const Gate &g, int M, size_t amp_bytes);

// ------------------------------------------------------------------- state
struct State {
    int M;
    qsim_prec prec;
    void *amps;
    bool owned;
    cudaStream_t stream;
    double *scratch;     // reduction partials; the last 4 doubles hold the result
    int scratch_blocks;  // partial slots (3 doubles each)
    cudaEvent_t ev;      // orders work across states' streams
    DevAllocator alloc;  // the device-memory functions the state was created with
};
inline size_t state_scratch_bytes(int slots) { return (3 * size_t(slots) + 4) * sizeof(double); }

inline size_t amp_bytes(qsim_prec p) { return p == QSIM_C64 ? 8 : 16; }

// ------------------------------------------------------ single-gate kernels
int launch_gate(void *amps, int M, qsim_prec prec, const Gate &g, cudaStream_t s);

// -------------------------------------------------------------- tile pass
// A pass holds a tile of 2^b amplitudes in shared memory: the L lowest qubits
// plus nh chosen higher qubits (hpos).  The remaining nout qubits (opos)
// number the tiles.  Every gate of the pass is applied to the tile in order.
constexpr int kMaxTileHigh = 8;
struct TilePassDesc {
    int b, L, nh, nout;
    int hpos[kMaxTileHigh];
    int opos[QSIM_MAX_QUBITS];
    int op_begin, op_count;
    int round_begin, round_count;  // register rounds (0 rounds: the shared-memory form)
    // register rounds: the pass's Hadamards are applied as (a + b, a - b) and
    // the product of their 1/sqrt(2) factors (a scalar, which commutes with
    // every op) once at the end, as pscale_hi + pscale_lo, when pscale_on
    int pscale_on;
    float pscale_hi, pscale_lo;
};

template <typename T2>
struct TileOp {
    T2 u[4];           // U00, U01, U10, U11 in the state precision (hi parts for complex64)
    T2 ul[4];          // lo parts (complex64; zero for complex128)
    uint32_t kind;     // Kind
    uint32_t tl;       // target position inside the tile (K_SCALE: unused)
    uint32_t lmask;    // control bits inside the tile (tile-local positions)
    uint32_t tab_off;  // K_DENSE: byte offset of a pre-phase table in the run buffer (0 = none)
    uint64_t gmask;    // control bits outside the tile (global positions)
    uint64_t gsel;     // K_SCALE: global target bit; K_PHRUN: byte offset of the record
    uint8_t npos;      // bits inserted to enumerate the touched amplitudes (or pairs)
    uint8_t pos[3];    // their tile-local positions, ascending
    uint8_t posval;    // bit k: the value inserted at pos[k]
    uint8_t tw;        // pre-phase table: index bits besides the target
    uint8_t tflags;    // bit 0: the table's target-0 entries are all exactly one
    uint8_t pad;
    uint8_t tpos[8];   // tile-local positions of the table's index bits
};
static_assert(sizeof(TileOp<float2>) % 16 == 0 && sizeof(TileOp<double2>) % 16 == 0, "ops are copied in 16-byte units");
// A pre-phase table holds, for every value of (tpos bits, target bit), the
// product of the diagonal factors of a run of phase gates that precedes an
// uncontrolled dense gate in a pass: entry (idx << 1) | target.  complex64:
// float4 (hi.re, hi.im, lo.re, lo.im) per entry; complex128: double2.

// A run of diagonal gates diag(e^{i a}, e^{i b}) with at most one control
// multiplies amplitude g by e^{i Phi(g)}, Phi a quadratic polynomial of the
// index bits: Phi = c0 + sum_q c[q] g_q + sum_{q<r} w[q][r] g_q g_r.  Phases
// are kept in turns as unsigned fixed point (2^32 per turn for complex64,
// 2^64 for complex128), so sums wrap exactly modulo 2 pi.  Device record,
// 16-byte aligned, at TileOp::gsel bytes into the plan's run buffer:
//   PhaseRunHdr; Turn c0; Turn c[M]; Turn w[M*M] (symmetric, zero diagonal);
//   then, at q_offset, Turn Q[2^b] = the quadratic part over the pass's tile
//   qubits, indexed by the tile-local index.
struct PhaseRunHdr {
    uint32_t M, b, q_offset, pad;  // q_offset: byte offset of Q from the record start
};
template <typename T2>
using TurnT = typename std::conditional<sizeof(T2) == 8, uint32_t, uint64_t>::type;

int launch_tile_pass(void *dst, const void *src, int M, qsim_prec prec, const TilePassDesc &d,
                     const void *ops_dev, const void *runs_dev, cudaStream_t s);

// Register rounds (complex64 tile passes with b = kRegThreadBits + RB): each
// of the block's 2^kRegThreadBits threads holds the 2^RB amplitudes of its
// index that differ in RB chosen tile qubits (the round's slot qubits) in
// registers and applies every gate of the round to them; shared memory is
// touched only between rounds, and the first (last) round reads (writes)
// device memory directly.
constexpr int kRegThreadBits = 8;  // 256 threads
struct RegOp {
    float2 u[4], ul[4];  // matrix, hi and lo parts (dense and diagonal kinds)
    uint32_t kind;       // K_DENSE, K_SWAPX, K_PHASE1, K_DIAG, K_SCALE, K_TAB, K_PHRUN
    uint32_t lmask;      // controls inside the tile (tile-local bits)
    uint64_t gmask;      // controls outside the tile
    uint64_t gsel;       // K_SCALE: outside target bit; K_PHRUN: record offset in the run buffer
    uint32_t tb;         // diagonal kinds: tile-local target bit; K_TAB: multiply only where this bit is set (0: all)
    uint32_t tab_off;    // K_TAB: byte offset of the table in the run buffer
    uint8_t k;           // pair kinds: slot bit of the target
    uint8_t tw;          // K_TAB: index bits
    uint16_t smask;      // slots the op touches (pair kinds: the lower slot of each pair)
    uint8_t tpos[12];    // K_TAB: tile-local positions of the index bits (bit j of the entry index)
    uint16_t cidx[16];   // K_TAB: index contribution of slot c (the slot bits among tpos; up to 9 index bits)
    uint32_t nmask;      // tile bits outside the slots that the thread's index must have set
    uint32_t tbn;        // K_DIAG: target bit when it is not a slot qubit (tested on the thread's index)
    uint16_t tsel;       // K_DIAG: slots whose target bit is set (target a slot qubit)
    uint8_t code;        // dispatch code of the register kernel (RegCode)
    uint8_t pad3;
    uint16_t pad2[2];
};
// Dispatch code of a RegOp: pair kinds by (kind, every pair touched, slot bit k).
enum RegCode : uint8_t {
    RC_DENSE = 0,     // + 4 * partial + k
    RC_RDENSE = 8,    // + 4 * partial + k
    RC_SWAP = 16,     // + 4 * partial + k
    RC_PHASE_ALL = 24,
    RC_PHASE = 25,
    RC_DIAG = 26,
    RC_SCALE = 27,
    RC_TAB = 28,
    RC_PHRUN = 29,
    RC_HAD = 32,      // + k: uncontrolled c [[1, 1], [1, -1]], the factor c deferred to the end of the pass
    RC_NHAD = 36,     // + k: uncontrolled real O = (H + E) / sqrt 2 with E small (a Hadamard with an error):
                      // (a + b + e00 a + e01 b, a - b + e10 a + e11 b) with e_j in u[j].x, 1/sqrt 2 deferred
};
static_assert(sizeof(RegOp) % 16 == 0, "RegOp is copied in 16-byte units");
struct RoundDesc {
    uint8_t pos[4];        // slot qubits (tile-local positions), ascending
    uint16_t op_begin;     // first op of the round, relative to the pass's first op
    uint16_t op_count;
};
int launch_tile_reg(void *dst, const void *src, int M, const TilePassDesc &d, const void *ops_dev,
                    const void *rounds_dev, const void *runs_dev, cudaStream_t s);
int tile_reg_prepare();
// Group one tile pass's ops into register rounds of RB slot qubits (plan.cu):
// appends to regops / rounds (and phase tables to runs); false if the pass
// cannot use them.
bool build_register_rounds(const std::vector<TileOp<float2>> &ops, int op_begin, int op_count, TilePassDesc &d,
                           int RB, std::vector<RegOp> &regops, std::vector<RoundDesc> &rounds,
                           std::vector<unsigned char> &runs);
// Specialised register passes (jit.cu): generate, compile (NVRTC) and load one
// kernel per pass; QSIM_EUNSUPPORTED (with *log) when NVRTC is unavailable.
// gathers[i], when present and non-null, is a qubit permutation (an
// involution) that pass i also applies to its input as it reads it.
int jit_build(const std::vector<const TilePassDesc *> &passes, const std::vector<const std::vector<int> *> &gathers,
              const std::vector<RegOp> &regops, const std::vector<RoundDesc> &rounds,
              const std::vector<unsigned char> &runs, std::vector<cudaLibrary_t> *libs,
              std::vector<cudaKernel_t> *kernels, std::string *log);
bool jit_available();  // NVRTC could be loaded
void jit_release(cudaLibrary_t lib);
void jit_release(const std::vector<cudaLibrary_t> &libs);
// The persistent trajectory kernel in register rounds ("qs_traj"): passes with
// their rounds, op j of pass p = regops[passes[p].op_begin + j] whose gate is
// trajectory op src[p][j]; `lanes` trajectories per CTA of 256 * lanes
// threads, __launch_bounds__(256 * lanes, min_blocks).
int jit_build_traj(int M, const std::vector<TilePassDesc> &passes, const std::vector<RegOp> &regops,
                   const std::vector<RoundDesc> &rounds, const std::vector<std::vector<int>> &src, int min_blocks,
                   int lanes, cudaLibrary_t *lib, cudaKernel_t *kernel, std::string *log);
size_t jit_pass_smem_bytes(const TilePassDesc &d);  // the two staged tiles of a specialised pass
size_t jit_traj_smem_bytes(const std::vector<TilePassDesc> &passes, int lanes);  // two-lane tile buffers (0: static)
int launch_jit_pass(cudaKernel_t k, void *dst, const void *src, int M, const TilePassDesc &d, const void *runs_dev,
                    cudaStream_t s);
constexpr int kTileOpSmemBytes = 24 * 1024;  // a pass's ops are staged in shared memory up to this size
int tile_max_bits(qsim_prec prec);
int tile_prepare(qsim_prec prec);  // one-time kernel attributes (call before any stream capture)

// ------------------------------------------------------------ fused blocks
// Geometry of one fused k-qubit block over a state of M qubits (see
// k_fused_tc.cu): tile qubits U = B u F (B the block, F the 7 lowest other
// qubits), tile-local index u = bits of U in ascending order.
// Fused tensor-core pass: tiles of 2^kFusedTileBits amplitudes, the k block
// qubits plus the 12 - k lowest other qubits; at most 2^kFusedRowBits
// sub-vectors per tile.
constexpr int kFusedTileBits = 12;
constexpr int kFusedRowBits = 9;
struct FusedDesc {
    int k;
    int unitary;                 // the block is unitary: rescale each sub-vector to its input norm
    int runbits;                 // qubits 0..runbits-1 are all in the tile: runs of 2^runbits amplitudes
    int nrb;                     // tile qubits above the run: 12 - runbits
    int rpos[kFusedTileBits];    // their device positions, ascending
    int nout;                    // qubits outside the tile (number the tiles)
    int opos[QSIM_MAX_QUBITS];
    int outsh;                   // staging swizzle: bits [0,4) of the tile index ^= bits [outsh, outsh+4)
    int direct;                  // sub-vectors 0..31 are amplitudes 0..31 of the tile: store without staging
    uint16_t posA[32];           // u of block combination a (sub-vector 0)
    uint16_t posM[1 << kFusedRowBits];  // u of sub-vector m (combination 0)
    uint8_t skew[32];            // split: lane l visits combination s ^ skew[l] at step s
    uint64_t runoff2[32];        // device offset of tile index 128 j (tile 0)
};
int fused_prepare();
size_t fused_rimg_halves(int k);  // FP16 values of one block's R_hi + R_lo image
// wait_ns bounds the kernel's pipeline waits (0 = 2 s); see k_fused_tc.cu.
int launch_fused(void *dst, const void *src, int M, const FusedDesc &d, const void *rimg_dev, int *status,
                 cudaStream_t s, uint64_t wait_ns);

// ------------------------------------------------------- qubit permutation
// out[pi(i)] = in[i] for an involution pi of the qubit positions (see
// k_perm.cu).  Tile qubits: spos[0..ns) ascending (they include 0..4);
// spi[j] = tile-local index of pi(spos[j]); outside qubits opos[0..nout)
// ascending and opi[j] = outside index of pi(opos[j]).
struct PermDesc {
    int ns, nout, lb;  // tile qubits, outside qubits, low qubits per contiguous run
    int sh;            // shared-memory swizzle: bits [0,4) of the local index ^= bits [sh, sh+4)
    int spos[12], spi[12];
    int opos[QSIM_MAX_QUBITS], opi[QSIM_MAX_QUBITS];
};
size_t perm_smem_bytes(const PermDesc &d, qsim_prec prec);  // at most 96 KiB
// Shared-memory wavefronts of one warp access: lane byte addresses, `width`
// (4, 8 or 16) bytes per lane.
int smem_wavefronts(const uint32_t *addr, int width);
int launch_perm(void *dst, const void *src, int M, qsim_prec prec, const PermDesc &d, cudaStream_t s);

// -------------------------------------------------------------- reductions
// Results land in scratch[result_offset .. +3): (norm, re <i|n>, im <i|n>).
int launch_reduce(const void *ideal, const void *noisy, int M, qsim_prec prec, double *scratch,
                  int scratch_blocks, cudaStream_t s);
int launch_probabilities(const void *amps, int M, qsim_prec prec, void *out, cudaStream_t s);
int launch_zero_state(void *amps, int M, qsim_prec prec, cudaStream_t s);
constexpr int kReduceSlots = 2048;  // max partial blocks

}  // namespace qs

// The opaque ABI handle is the internal state record.
struct qsim_state : qs::State {};

namespace qs {
// Plan creation whose device tables are allocated stream-ordered on
// alloc_stream (nullptr: plain cudaMalloc) through `alloc` (nullptr: the
// functions in force now), and release without a device synchronisation: the
// caller guarantees that the plan's work has completed or is ordered before
// alloc_stream's later work.
int plan_create_on(int M, qsim_prec prec, const qsim_gate *gates, size_t n, const qsim_opts *opts,
                   cudaStream_t alloc_stream, const DevAllocator *alloc, qsim_plan **out);
void plan_release(qsim_plan *p);
}  // namespace qs
