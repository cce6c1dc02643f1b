/*
 * qsim.h -- C ABI of the GB300 error-injecting state-vector simulator.
 *
 * What the library computes (Obenland & Despain, "A Parallel Quantum Computer
 * Simulator"):
 *   - Section 1.2: an M-qubit register is a vector of 2^M complex amplitudes;
 *     the index of an amplitude is the bit value of its basis state (qubit q =
 *     bit q of the index, bit 0 least significant); the probability of a
 *     state is |amplitude|^2.
 *   - Section 1.3: a gate is a 2^M x 2^M matrix times that vector.
 *   - Section 2.1 (Figure 3): a gate on one target bit is a 2x2 operation on
 *     every pair of states whose indices differ only in that bit; a
 *     controlled gate (Table 1 / Figure 2, Section 2.0's one-, two- and
 *     three-bit controlled-NOTs) applies it only where all control bits are 1.
 *   - Sections 1.4 / 2.0: operational errors are deviations of the rotation
 *     angles; the library applies gates that already carry their errors, and
 *     builds erroneous gates itself for error trajectories.
 *   - Fidelity of the noisy state against the error-free state:
 *     F = |<ideal|noisy>|^2 (not renormalised) with the noisy norm beside it.
 *
 * Conventions for every entry point:
 *   - Return value: QSIM_OK (0) or a negative QSIM_E* code.  On an error the
 *     thread-local message of qsim_last_error() says what failed; no output is
 *     written.  QSIM_ECUDA means a CUDA call failed; after a sticky device
 *     error every later call fails too.
 *   - Amplitudes are interleaved complex numbers (re, im): float pairs for
 *     QSIM_C64, double pairs for QSIM_C128, index order as above.
 *   - Host arrays passed in (gates, matrices, error angles) are read during
 *     the call and may be freed when it returns; the caller owns them.
 *     Output buffers belong to the caller.
 *   - Work on a state runs on that state's CUDA stream (qsim_set_stream;
 *     default: the legacy default stream), in call order.  Calls that return
 *     host values wait for that stream; the others return once the work is
 *     queued.
 *   - Nothing here is thread-safe for one state or plan used from several
 *     host threads at once; distinct states and plans are independent.
 */
#ifndef QSIM_H_
#define QSIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define QSIM_OK 0
#define QSIM_EINVAL (-1)      /* bad argument: qubit out of range, repeated qubit, bad M, ... */
#define QSIM_ENOMEM (-2)      /* device allocation failed or over the budget */
#define QSIM_ECUDA (-3)       /* a CUDA call failed */
#define QSIM_ETIMEOUT (-4)    /* a bounded device wait ran out */
#define QSIM_EBUSY (-5)       /* the serving queue is full */
#define QSIM_EUNSUPPORTED (-6)/* a valid request this build does not handle */

/* Largest qubit count accepted (2^34 complex64 amplitudes = 128 GiB). */
#define QSIM_MAX_QUBITS 34

typedef enum { QSIM_C64 = 0, QSIM_C128 = 1 } qsim_prec;

/* One gate (Section 2.0): a 2x2 complex matrix U applied to the target qubit
 * where every control qubit is 1 (Section 2.1).  U is row-major with
 * interleaved real and imaginary parts: U00re, U00im, U01re, U01im, U10re,
 * U10im, U11re, U11im.  X, CNOT and Toffoli are U = X with 0, 1 or 2
 * controls; a rotation gate carries its (erroneous) angle inside U.
 * 80 bytes, no padding. */
typedef struct qsim_gate {
    double U[8];
    int32_t target;
    int32_t ncontrols;   /* 0, 1 or 2 */
    int32_t controls[2]; /* distinct, != target; entries past ncontrols are ignored */
} qsim_gate;

/* How a circuit is executed.  Every mode computes the same gates in the same
 * order; they differ in how many gates one pass over the state vector applies. */
typedef enum {
    QSIM_MODE_AUTO = 0,     /* complex64 with M >= 20: the tile passes or the fused blocks, whichever a
                             * time model of the planned passes predicts faster (qsim_plan_describe
                             * prints the estimates); otherwise the tile passes */
    QSIM_MODE_UNFUSED = 1,  /* one kernel launch per gate */
    QSIM_MODE_TILED = 2,    /* shared-memory tiles: many gates per pass over the vector */
    QSIM_MODE_FUSED = 3     /* runs of gates merged into dense 2^k x 2^k blocks (tensor cores) */
} qsim_mode;

typedef struct qsim_opts {
    int32_t mode;       /* qsim_mode */
    int32_t fuse_k;     /* QSIM_MODE_FUSED block width 2..5 (2 runs as 3); 0 = default (5).  The fused
                         * mode needs complex64 and M >= 12, and falls back to TILED otherwise */
    int32_t tile_bits;  /* QSIM_MODE_TILED tile size 2^tile_bits amplitudes, 6..13; 0 = default */
    int32_t use_graph;  /* 1: a plan replays its launches as one captured CUDA graph */
    int32_t specialize; /* 1: each complex64 register tile pass is generated as its own kernel (op kinds,
                         * masks and matrix entries as constants) and compiled with NVRTC at plan
                         * creation: slower creation (about a second), faster execution, same
                         * results; without NVRTC the plan keeps the general kernel */
    int32_t wait_us;    /* QSIM_MODE_FUSED: bound of the tensor-core kernel's pipeline waits, in
                         * microseconds; 0 = 2 s.  A wait that runs out stops the kernel (the CTA
                         * drains its copies and MMAs in flight, with the full 2 s bound, and
                         * frees its tensor memory) and qsim_plan_status then reports
                         * QSIM_ETIMEOUT; the state is undefined.  For failure-detection tests */
    int32_t subspace;   /* 1: the plan applies the circuit to |0...0> (the input of qsim_plan_execute is
                         * not read; dst is overwritten) and runs each gate only on the amplitudes
                         * the qubits touched so far can make nonzero (Section 3.2, Figure 7: state
                         * values are allocated once a gate first uses their qubit; EQ 6): qubits
                         * are renumbered in the order gates first touch them, gates with a control
                         * no gate has touched are left out, and the gates between two first touches
                         * run, in `mode`, on the first 2^(qubits touched) amplitudes; at the end at
                         * most two in-place permutation passes restore the qubit order.  The result
                         * equals the flat plan's up to rounding.  qsim_plan_describe lists the
                         * segments.  Per-launch timing (qsim_plan_set_timing) is not recorded */
} qsim_opts;

/* Counts describing one execution of a plan. */
typedef struct qsim_plan_stats {
    int64_t n_gates;       /* gate records in the circuit */
    int64_t n_passes;      /* passes over the whole state vector (an in-place execution) */
    int64_t n_launches;    /* kernel launches per in-place execution; an out-of-place execution whose
                            * first specialised pass gathers the front permutation (see
                            * qsim_plan_execute) launches one fewer */
    int32_t mode;          /* the mode actually used */
    int32_t tile_bits;     /* tile size used (QSIM_MODE_TILED) */
    int32_t fuse_k;        /* block width used (QSIM_MODE_FUSED) */
    int32_t n_blocks;      /* fused blocks (QSIM_MODE_FUSED) */
    double algo_bytes;     /* algorithmic device-memory bytes (read + write) per execution */
    double amp_updates;    /* n_gates * 2^M */
    int64_t table_bytes;   /* device bytes of the plan's tables (gate ops, rounds, phase runs, fused
                            * matrices), copied from the host when the plan is created */
} qsim_plan_stats;

typedef struct qsim_state qsim_state;   /* opaque; owned by the library */
typedef struct qsim_plan qsim_plan;     /* opaque; owned by the library */

/* -------------------------------------------------------------- states */

/* Allocate a 2^M-amplitude state on the current CUDA device and set it to
 * |0...0> (Section 1.2, Figure 1(a)).  M in [1, QSIM_MAX_QUBITS].
 * QSIM_ENOMEM if the device has no room. */
int qsim_alloc(int M, qsim_prec prec, qsim_state **out);

/* Use caller-owned device memory (2^M amplitudes, 16-byte aligned) as a
 * state, without initialising it.  The memory must outlive the state;
 * qsim_free leaves it alone. */
int qsim_wrap(void *device_amps, int M, qsim_prec prec, qsim_state **out);

/* Release a state (and its amplitudes if qsim_alloc made them).  NULL is a
 * no-op.  Waits for the state's stream first. */
void qsim_free(qsim_state *st);

/* Run the state's work on this cudaStream_t (NULL = legacy default stream). */
int qsim_set_stream(qsim_state *st, void *cuda_stream);

/* M, precision and device address of the amplitudes. Any output may be NULL. */
int qsim_state_info(const qsim_state *st, int *M, int *prec, void **device_amps);

/* |0...0> */
int qsim_reset(qsim_state *st);

/* Copy 2^M amplitudes in from `amps` (host memory, or device memory if
 * on_device != 0).  Host copies wait for the state's stream. */
int qsim_set_state(qsim_state *st, const void *amps, int on_device);

/* As qsim_set_state, but only queues the copy on the state's stream and
 * returns (outside the paper; for pipelines that copy the next input while
 * the current one is being simulated).  Host memory should be page-locked
 * (cudaHostAlloc / pinned) for the copy to run asynchronously, and `amps` must
 * stay unchanged until the state's stream has passed the copy: until a later
 * call that waits for the state (qsim_get_state, qsim_fidelity, ...) or a
 * stream synchronisation.  Work queued on the state afterwards, on any
 * stream, is ordered after the copy as usual. */
int qsim_set_state_async(qsim_state *st, const void *amps, int on_device);

/* Copy the 2^M amplitudes out to `amps` (host, or device if on_device != 0).
 * Host copies wait for the state's stream. */
int qsim_get_state(const qsim_state *st, void *amps, int on_device);

/* dst := src (same M and precision), on dst's stream after src's queued work. */
int qsim_copy_state(qsim_state *dst, const qsim_state *src);

/* --------------------------------------------------------------- gates */

/* Apply one gate (Section 2.1, Figure 3): for every index i with bit `target`
 * 0 and all control bits 1, (a_i, a_j) <- U (a_i, a_j), j = i | 2^target.
 * U as in qsim_gate.  QSIM_EINVAL for an out-of-range or repeated qubit,
 * ncontrols outside 0..2, or a non-finite U. */
int qsim_apply_gate(qsim_state *st, const double U[8], int target,
                    const int *controls, int ncontrols);

/* Apply n gates in order (Section 2.0: a circuit given as logic gates).
 * opts may be NULL (QSIM_MODE_AUTO).  Equivalent to qsim_plan_create +
 * qsim_plan_execute(plan, st, NULL) + qsim_plan_destroy. */
int qsim_apply_circuit(qsim_state *st, const qsim_gate *gates, size_t n,
                       const qsim_opts *opts);

/* ---------------------------------------------------------------- plans */

/* Check and compile a circuit for states of M qubits and one precision:
 * classify gates, group them into passes or fused blocks, build the fused
 * matrices (FP64 products rounded once to the state precision) and copy the
 * tables to the device.  The plan may be executed any number of times. */
int qsim_plan_create(int M, qsim_prec prec, const qsim_gate *gates, size_t n,
                     const qsim_opts *opts, qsim_plan **out);

/* dst := circuit(src).  src == NULL or src == dst runs in place; otherwise
 * src is left untouched (same M and precision).  Runs on dst's stream after
 * src's queued work.  In QSIM_MODE_TILED, runs of SWAP gates (each three
 * CNOTs) are planned as one qubit permutation at the front of the circuit,
 * the later gates relabelled; when that permutation is an involution and the
 * plan is specialised, an out-of-place execution applies it inside the first
 * pass's reads instead of a separate permutation pass. */
int qsim_plan_execute(const qsim_plan *plan, qsim_state *dst, const qsim_state *src);

int qsim_plan_stats_get(const qsim_plan *plan, qsim_plan_stats *out);

/* A text description of the plan's passes (outside the paper; for tests and
 * tuning): one line per pass (kind, tile qubits, op and round counts) and,
 * for register tile passes, one line per round (slot qubits, each op's kind).
 * Writes at most len - 1 characters and a terminating NUL into buf (buf may be
 * NULL when len is 0); *needed (may be NULL) = the full length + 1. */
int qsim_plan_describe(const qsim_plan *plan, char *buf, int64_t len, int64_t *needed);

/* Wait for the device and report whether any kernel of this plan gave up a
 * bounded wait since the last call: QSIM_OK, or QSIM_ETIMEOUT (the affected
 * state is then undefined).  Clears the record. */
int qsim_plan_status(const qsim_plan *plan);

/* Release a plan; NULL is a no-op.  Waits for the device. */
void qsim_plan_destroy(qsim_plan *plan);

/* Per-launch timing, for profiling.  While enabled (enable != 0), every
 * qsim_plan_execute records a CUDA event before its first launch and after
 * each launch, on dst's stream, without waiting.  Timing is ignored for
 * executions replayed from a CUDA graph. */
int qsim_plan_set_timing(qsim_plan *plan, int enable);

/* Wait for the recorded events and report, for each launch index j < n_max
 * of one execution: ms[j] = milliseconds summed over the timed executions,
 * bytes[j] = algorithmic bytes of that launch, kind[j] = 0 single gate,
 * 1 shared-memory tile pass, 2 fused block, 3 qubit permutation pass,
 * 4 register tile pass (complex64), 5 specialised register tile pass,
 * 6 a permutation pass left out by the last execution (the next pass gathered
 * it; no launch, bytes 0).
 * *executions = number of timed executions.
 * Any output array may be NULL.  Clears the record. */
int qsim_plan_timing(qsim_plan *plan, int64_t n_max, double *ms, double *bytes, int32_t *kind,
                     int64_t *executions);

/* ------------------------------------------------------------ reductions */

/* F = |sum_i conj(ideal_i) noisy_i|^2 and norm_noisy = sum_i |noisy_i|^2,
 * accumulated in FP64 in a fixed order (deterministic).  Runs on noisy's
 * stream after ideal's queued work; waits for it.  F or norm_noisy may be
 * NULL.  Both states must have equal M and precision. */
int qsim_fidelity(const qsim_state *ideal, const qsim_state *noisy,
                  double *F, double *norm_noisy);

/* The sums behind qsim_fidelity: out[0] = sum_i |noisy_i|^2, out[1] + i out[2]
 * = sum_i conj(ideal_i) noisy_i, same order and accumulation.  For a state
 * split over ranks (qsim_shard_plan_create) each rank's three sums add up to
 * the whole state's (an all-reduce of 3 doubles; EQ 3's global sum); then
 * F = out[1]^2 + out[2]^2.  Waits for noisy's stream. */
int qsim_overlap(const qsim_state *ideal, const qsim_state *noisy, double out[3]);

/* norm = sum_i |a_i|^2 (Section 1.2), FP64 accumulation. */
int qsim_norm(const qsim_state *st, double *norm);

/* p_i = |a_i|^2 for all 2^M states (Section 1.2, Figure 1) into `out`:
 * float for QSIM_C64, double for QSIM_C128; host memory, or device memory if
 * on_device != 0. */
int qsim_probabilities(const qsim_state *st, void *out, int on_device);

/* Fidelity and norm for callers that cannot allocate device memory.  The
 * paper has no counterpart: this entry point exists for code that must not
 * call cudaMalloc -- plugins whose host application owns all GPU memory
 * through its own pool, latency-critical loops that must never enter the
 * allocator -- and so cannot create the qsim_state that qsim_fidelity needs.
 *
 * ideal_amps, noisy_amps: caller-owned device arrays of 2^M amplitudes
 * (16-byte aligned; ideal_amps may be NULL for the norm alone, F is then 0).
 * Computes the same F = |sum conj(ideal_i) noisy_i|^2 and norm_noisy =
 * sum |noisy_i|^2 as qsim_fidelity, on cuda_stream (NULL = legacy default),
 * then copies the result to the host and waits for that stream.  Allocates
 * nothing: its scratch is one fixed 1.5 MiB device array that every GPU which
 * loads the library holds until the process exits, so M is limited to
 * [1, 32]; larger M returns QSIM_EINVAL with a message.  The first call on a
 * device looks the array's address up (cudaGetSymbolAddress) and keeps it for
 * the life of the process (a cudaDeviceReset in between is not supported);
 * that first call should come before any stream capture.  All calls share
 * the array and it keeps the last call's values; calls whose work overlaps
 * on the GPU (other streams or host threads) race on it. */
int qsim_fidelity_noalloc(const void *ideal_amps, const void *noisy_amps, int M, qsim_prec prec,
                          void *cuda_stream, double *F, double *norm_noisy);

/* --------------------------------------------------------- trajectories */

typedef struct qsim_traj_opts {
    int32_t fuse_k;     /* reserved for fused blocks: 0 or 1 (one gate at a time) */
    int32_t use_graph;  /* 1: each run replays a captured CUDA graph */
    int32_t kernel;     /* 0: autotuned; 1: shared-memory tile kernel; 2: register-round kernel
                         * generated for the circuit (NVRTC; falls back to 1 without it) */
    int32_t reserved;
} qsim_traj_opts;

typedef struct qsim_traj_plan qsim_traj_plan;  /* opaque; owned by the library */

/* Compile a circuit for up to max_T error trajectories (complex64, M in
 * [1, 20]): computes the error-free state, allocates the per-CTA workspaces
 * and picks the kernel configuration by timing the candidates on a short
 * batch (cached per circuit in the process): the shared-memory tile kernel
 * with tiles of 2^10..2^13 amplitudes, and the register-round kernel
 * generated for the circuit with 3 or 4 register qubits per thread (the
 * fusion width of a round) and 1 or 2 resident trajectories per SM.  The plan
 * owns its own CUDA stream. */
int qsim_traj_plan_create(int M, const qsim_gate *ideal, const double *err_axis, size_t n, int max_T,
                          const qsim_traj_opts *opts, qsim_traj_plan **out);

/* Run T <= max_T trajectories with errors eps (T x n doubles, host) in one
 * persistent kernel launch (replayed from a CUDA graph when use_graph is set);
 * outputs as for qsim_run_trajectories.  Synchronous. */
int qsim_traj_plan_run(qsim_traj_plan *plan, const double *eps, int T, double *F_out, double *mean,
                       double *var);

/* Tile size chosen, tile passes per trajectory and the persistent grid size. */
int qsim_traj_plan_info(const qsim_traj_plan *plan, int *tile_bits, int *n_passes, int *grid);

/* A text description of the chosen kernel and the autotuner's timings of the
 * candidates (outside the paper; for tuning).  Writes at most len - 1
 * characters and a NUL into buf (NULL when len is 0); *needed (may be NULL)
 * = the full length + 1. */
int qsim_traj_plan_describe(const qsim_traj_plan *plan, char *buf, int64_t len, int64_t *needed);

void qsim_traj_plan_destroy(qsim_traj_plan *plan);

/* T error trajectories of one circuit (Sections 1.4, 2.0: every gate's angle
 * deviates), all started from |0...0>, in one persistent kernel launch
 * (qsim_traj_plan_create + qsim_traj_plan_run + qsim_traj_plan_destroy).
 * Gate g of trajectory t is U_g . exp(-i eps[t*n+g]/2 (axis_g . sigma)),
 * built on the device in FP64; axis_g = (0,0,0) means gate g takes no error.
 * err_axis: n x 3 doubles; eps: T x n doubles (host).  F_out[t] (host, T
 * doubles, may be NULL) receives each trajectory's fidelity against the
 * error-free run; *mean and *var (may be NULL) the mean and unbiased
 * variance of F.  complex64 amplitudes, M in [1, 20].  Synchronous. */
int qsim_run_trajectories(int M, const qsim_gate *ideal, const double *err_axis, size_t n,
                          const double *eps, int T, const qsim_traj_opts *opts,
                          double *F_out, double *mean, double *var);

/* -------------------------------------------------------------- serving */

/* A request loop with continuous batching.  A request is one simulation as
 * the paper runs it (Section 2.0): M qubits from |0...0>, the error-free
 * gates and the erroneous gates applied to two complex64 copies, then F and
 * the noisy norm (qsim_fidelity).  A scheduler thread admits the oldest
 * waiting request as soon as a slot is free and its two state vectors fit in
 * hbm_budget; each slot runs on its own CUDA stream, so admitted requests
 * overlap on the device.  Results do not depend on the mix. */
typedef struct qsim_server qsim_server;  /* opaque; owned by the library */

typedef struct qsim_server_opts {
    uint64_t hbm_budget;  /* bytes of state vectors held at once (2 x 2^M x 8 per request) */
    int32_t max_slots;    /* requests in flight at once, 1..256 */
    int32_t mode;         /* qsim_mode of the requests' circuits */
} qsim_server_opts;

typedef struct qsim_request_result {
    uint64_t id;
    int32_t status;      /* QSIM_OK; QSIM_ENOMEM if the request can never fit the budget */
    int32_t M;
    int32_t n_gates;
    int32_t pad;
    double F, norm;      /* |<ideal|noisy>|^2 and the noisy norm */
    double t_submit, t_start, t_done;  /* seconds on the server's clock */
} qsim_request_result;

typedef struct qsim_server_stats {
    uint64_t n_submitted, n_completed, n_pending;
    uint64_t bytes_in_use, peak_bytes;  /* state-vector bytes held now / at most */
    int32_t max_active;                 /* most requests in flight at once */
    int32_t pad;
    double now;                         /* the server's clock, seconds */
} qsim_server_stats;

/* Start a server on the current device (its own memory pool and streams). */
int qsim_server_create(const qsim_server_opts *opts, qsim_server **out);

/* Queue a request: n gates of the error-free circuit and n of the erroneous
 * one (copied; checked now, QSIM_EINVAL on a bad gate).  QSIM_EBUSY if 2^20
 * requests are already waiting.  *id identifies its result. */
int qsim_server_submit(qsim_server *srv, int M, const qsim_gate *ideal, const qsim_gate *noisy, size_t n,
                       uint64_t *id);

/* Move up to max finished results into out (completion order), waiting up to
 * wait_ms for the first one; *nout = how many. */
int qsim_server_poll(qsim_server *srv, qsim_request_result *out, int max, int *nout, int wait_ms);

int qsim_server_get_stats(qsim_server *srv, qsim_server_stats *out);

/* Finish every queued request, then stop and release everything.  Results
 * not polled are dropped. */
void qsim_server_destroy(qsim_server *srv);

/* ------------------------------------------------------ device memory */

/* Device-memory hook (outside the paper; a deployment matter: the library's
 * state vectors and tables can then live in the caller's memory pool, e.g.
 * a framework's caching allocator, instead of next to it).
 *
 * alloc(bytes, cuda_stream, ctx) returns `bytes` of device memory on the
 * current device, 256-byte aligned, or NULL when it has none (the library
 * call then fails with QSIM_ENOMEM).  cuda_stream is the stream on which the
 * library first uses the memory (NULL = legacy default stream); a
 * stream-ordered allocator may hand out memory whose earlier users are
 * ordered before that stream's later work.  free(ptr, bytes, cuda_stream,
 * ctx) gives it back: the library's work on ptr is queued on cuda_stream (or
 * already complete) when free is called.
 *
 * Every device allocation the library makes after this call goes through the
 * pair: qsim_alloc's amplitudes and every state's reduction scratch, plan
 * tables, trajectory-plan workspaces, and the server's state vectors and
 * scratch (the server then leaves its own memory pool unused; its HBM budget
 * still counts the bytes).  Each state, plan, trajectory plan and server
 * keeps the pair it was created with and releases its memory through it, so
 * the functions and ctx must stay valid until every object created under
 * them is released.  Not routed: pinned host staging buffers, and the module
 * memory of kernels compiled at plan creation (NVRTC), which the CUDA driver
 * allocates.  alloc = free = NULL restores the CUDA runtime (cudaMalloc /
 * cudaMallocAsync).  QSIM_EINVAL if exactly one of the two is NULL.  The
 * hook may be called from the server's scheduler thread. */
typedef void *(*qsim_device_alloc_fn)(size_t bytes, void *cuda_stream, void *ctx);
typedef void (*qsim_device_free_fn)(void *ptr, size_t bytes, void *cuda_stream, void *ctx);
int qsim_set_allocator(qsim_device_alloc_fn alloc, qsim_device_free_fn free, void *ctx);

/* ------------------------------------------------------------- qutrits */

/* The three-state model (Section 2.0: the detailed model with a third,
 * temporary level per particle, 3^M states; Sections 3.0-3.1).  The
 * amplitudes of M three-level particles are 3^M complex numbers, the index
 * written in base 3 with digit q = the level of particle q (digit 0 least
 * significant).  A transformation is a 3x3 matrix U (row-major, re/im
 * interleaved: 18 doubles) on a target particle, applied to every triple of
 * states differing only in the target's level, (a_i, a_{i+3^t}, a_{i+2 3^t})
 * for each i with digit t = 0, where each control particle controls[k] is at
 * level levels[k].  168 bytes, no padding. */
typedef struct qsim_gate3 {
    double U[18];
    int32_t target;
    int32_t ncontrols;   /* 0, 1 or 2 */
    int32_t controls[2]; /* distinct particles, != target */
    int32_t levels[2];   /* 0, 1 or 2 */
} qsim_gate3;

/* Apply n transformations in order to caller-owned device amplitudes (3^M
 * interleaved complex numbers, 16-byte aligned), on cuda_stream (NULL =
 * legacy default), one kernel launch each; returns once queued.  M in
 * [1, 21].  QSIM_EINVAL for an out-of-range particle or level, a repeated
 * particle, or a non-finite matrix (nothing is queued then). */
int qsim_qutrit_apply(void *device_amps, int M, qsim_prec prec, const qsim_gate3 *gates, size_t n,
                      void *cuda_stream);

/* out[0] = sum |noisy_i|^2, out[1] + i out[2] = sum conj(ideal_i) noisy_i over
 * the 3^M amplitudes (FP64, fixed order); ideal_amps may be NULL (then out[1]
 * = out[2] = 0).  F = out[1]^2 + out[2]^2.  Allocates 3^M / 2^16 x 24 bytes of
 * device scratch for the call; waits for cuda_stream. */
int qsim_qutrit_overlap(const void *ideal_amps, const void *noisy_amps, int M, qsim_prec prec, void *cuda_stream,
                        double out[3]);

/* ---------------------------------------------------------- decoherence */

/* A circuit with decoherence after every operation (Section 3.4: two more
 * transformations after each operation and a sum over the whole state; EQ 3,
 * EQ 8).  The paper leaves the transformations open; this library's reading:
 * after gate g on target t (applied where its controls are 1),
 *   1. dephasing: Rz(delta[g]) = diag(e^{-i delta/2}, e^{+i delta/2}) on t
 *      (on every amplitude);
 *   2. amplitude damping on t as a quantum jump: with P1 = the summed |a|^2
 *      of t's 1 states and N = the norm, p = gamma P1 / N; if r[g] < p the
 *      jump operator [[0, sqrt(gamma)], [0, 0]] is applied, otherwise the
 *      no-jump operator diag(1, sqrt(1 - gamma)), each scaled so that the
 *      norm stays N.
 * The state is updated in place on its stream; delta (radians) and r
 * (uniform draws in [0, 1)) are n doubles each, chosen by the caller (seeded),
 * so runs are reproducible.  jumps[g] (n int32, may be NULL) receives 1 where
 * the jump was taken and p_out[g] (n doubles, may be NULL) the probability p;
 * the sums are FP64 and in a fixed order.  One pass over the state per
 * operation: the damping of operation g is applied in the pass of gate g + 1.
 * gamma in [0, 1]; QSIM_EINVAL for a bad gate or a non-finite delta or r.
 * Allocates 32 KiB + 12 n bytes of device scratch for the call.  Waits for
 * the state's stream. */
int qsim_run_decoherence(qsim_state *st, const qsim_gate *gates, size_t n, const double *delta, const double *r,
                         double gamma, int32_t *jumps, double *p_out);

/* ------------------------------------------------------------- sharding */

/* One state over P = 2^n_global ranks (Section 3.1; Section 3.3, Figure 8):
 * the values of n_global qubits (initially the top ones, M - n_global ..
 * M - 1) select the rank that holds an amplitude; each rank holds the
 * 2^L amplitudes (L = M - n_global) of its rank bits as an L-qubit state,
 * local qubit s = bit s of the local index.  The plan (host records only, no
 * device work) lists, for one rank, the steps that apply the circuit:
 *   kind 0: gates on the local state (qsim_shard_step_gates; run them with a
 *           plan of L qubits).  A gate controlled by a rank bit that is 0 on
 *           this rank is left out, a control on a rank bit that is 1 is
 *           dropped, and a diagonal gate on a rank-bit target becomes the
 *           factor of this rank's bit;
 *   kind 1: a redistribution of n_pairs qubits (global_bits[i] = the rank bit
 *           j_i of pair i): with C = 2^(L - n_pairs) and the local state cut
 *           into chunks of C amplitudes (chunk b = the values of the top
 *           n_pairs local bits, bit i of b for pair i), this rank exchanges,
 *           for every b other than its own bits (rank >> j_i) & 1, its chunk b
 *           with the same-sized chunk of the rank whose bits j_i equal b and
 *           whose other bits equal this rank's (the partner's chunk b' = this
 *           rank's own index): send chunk b, receive into chunk b.  Afterwards
 *           the top local qubit L - n_pairs + i and rank bit j_i have traded
 *           their logical qubits.
 * A redistribution is planned only when a non-diagonal gate targets a qubit
 * held in a rank bit: that qubit trades places with the local qubit whose next
 * use as such a target lies furthest ahead (the same choice on every rank).
 * With restore_order != 0 the plan ends in the starting layout (logical
 * qubit q at local bit q, or at rank bit q - L).  Rank in [0, 2^n_global),
 * n_global in [0, min(M - 1, 20)]. */
typedef struct qsim_shard_plan qsim_shard_plan;
int qsim_shard_plan_create(int M, int n_global, int rank, const qsim_gate *gates, size_t n, int restore_order,
                           qsim_shard_plan **out);
/* Steps, redistributions, and the sum over redistributions of the fraction
 * of a shard each rank sends (1 - 2^-n_pairs each; EQ 2's reorganised blocks
 * over all blocks).  Any output may be NULL. */
int qsim_shard_plan_info(const qsim_shard_plan *p, int64_t *n_steps, int64_t *n_exchanges, double *moved);
/* Step i: kind (0 local gates, 1 redistribution), its gate count, its pair
 * count and the rank bits of the pairs (global_bits: room for n_global ints;
 * may be NULL).  Any output may be NULL. */
int qsim_shard_step(const qsim_shard_plan *p, int64_t i, int *kind, int64_t *n_gates, int *n_pairs,
                    int *global_bits);
/* The local gates of step i (qubits numbered 0 .. L-1) into out[0 .. n_gates). */
int qsim_shard_step_gates(const qsim_shard_plan *p, int64_t i, qsim_gate *out, size_t cap);
void qsim_shard_plan_destroy(qsim_shard_plan *p);

/* ----------------------------------------------------------- autotuning */

/* The tuning cache (outside the paper; execution choices, not results).
 * QSIM_MODE_AUTO picks among tile passes of 2^12 or 2^11 amplitudes and fused
 * blocks of width 5, 4 or 3 by a time model of the planned passes whose rates
 * are measured on the device (a light and a heavy tile pass, a permutation
 * pass, one fused block of each width on and off qubits 0..4, on a 26-qubit
 * state: about a second, once per device, precision and tile-kernel kind);
 * trajectory plans time their candidate kernels on a short batch.  Both are
 * kept in memory and, when a cache file is set, in that JSON file, which later
 * processes read instead of measuring again.  path = NULL keeps them in memory
 * only (the default unless the environment variable QSIM_TUNE_CACHE names a
 * file).  Setting the path drops what is in memory. */
int qsim_tune_set_cache(const char *path);

/* The measured rates AUTO uses for this precision and tile-kernel kind
 * (specialize != 0: the NVRTC-generated passes), measuring them now unless
 * the cache holds them, as a JSON object in buf (at most len - 1 characters
 * and a NUL; *needed = the full length + 1): bandwidths in bytes/s, the FMA
 * rate in FMA-equivalents/s, and where they came from. */
int qsim_tune_rates(int prec, int specialize, char *buf, int64_t len, int64_t *needed);

/* ---------------------------------------------------------------- misc */

/* Message of the last failed call on this host thread ("" if none). */
const char *qsim_last_error(void);

/* Library version string. */
const char *qsim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_H_ */
