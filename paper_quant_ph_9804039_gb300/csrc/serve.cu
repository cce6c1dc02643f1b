// Serving: a request loop with continuous batching.
//
// A request is one error-injecting simulation as the paper runs it (Section
// 2.0): an M-qubit register starts in |0...0>, the error-free circuit and the
// circuit with injected errors are applied to two copies, and the fidelity
// |<ideal|noisy>|^2 and the noisy norm come back.  Requests of different
// qubit counts and lengths arrive at any time; a native scheduler thread
// admits the oldest waiting request as soon as an execution slot is free and
// its two state vectors (2 x 2^M complex64) fit in the device-memory budget.
// Each slot runs its request on its own CUDA stream, so requests admitted
// together overlap on the device; every allocation and release is
// stream-ordered (a private memory pool for the states, cudaMallocAsync for
// the plans' tables), so admitting or retiring one request never waits for
// the others.  A host callback on the slot's stream stamps the completion
// time and wakes the scheduler.  A request's kernels, launch shapes and
// reduction order do not depend on what else runs, so its result is the same
// alone and in any mix.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "qsim_internal.h"

using namespace qs;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id;
    int M;
    std::vector<qsim_gate> ideal, noisy;
    double t_submit;
};

struct Slot {
    qsim_server *srv = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    double *scratch = nullptr;  // reduction partials + result
    double *h_res = nullptr;    // pinned copy of (norm, re, im)
    bool busy = false;
    Request req;
    void *amps[2] = {nullptr, nullptr};
    qsim_plan *plans[2] = {nullptr, nullptr};
    size_t bytes = 0;
    double t_start = 0;
    std::atomic<int> done{0};
    std::atomic<double> t_done{0};
    int status = QSIM_OK;
};

}  // namespace

struct qsim_server {
    qsim_server_opts opts{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work;  // wakes the scheduler
    std::condition_variable cv_done;  // wakes pollers
    std::deque<Request> pending;
    std::deque<qsim_request_result> done;
    std::vector<Slot *> slots;
    size_t bytes_in_use = 0, peak_bytes = 0;
    uint64_t next_id = 1;
    uint64_t n_submitted = 0, n_completed = 0;
    int max_active = 0;
    bool stop = false;
    cudaMemPool_t pool = nullptr;  // used when no allocator hook was set at creation
    DevAllocator alloc{};          // the hook in force at creation, if any
    std::thread worker;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

constexpr size_t kMaxPending = size_t(1) << 20;

void CUDART_CB on_slot_done(void *arg) {
    Slot *s = static_cast<Slot *>(arg);
    s->t_done.store(s->srv->now());
    s->done.store(1);
    std::lock_guard<std::mutex> lock(s->srv->mu);
    s->srv->cv_work.notify_all();
}

size_t request_bytes(int M) { return 2 * (size_t(1) << M) * sizeof(float) * 2; }

// Queue the whole request on the slot's stream (called by the scheduler).
int start_request(qsim_server *srv, Slot *s) {
    const Request &r = s->req;
    const size_t vec = (size_t(1) << r.M) * 8;
    for (int k = 0; k < 2; ++k) {
        if (srv->alloc.alloc) {
            if (int rc = dmalloc(srv->alloc, &s->amps[k], vec, s->stream, "served state")) return rc;
        } else {
            QS_CUDA(cudaMallocFromPoolAsync(&s->amps[k], vec, srv->pool, s->stream));
        }
    }
    qsim_opts po{srv->opts.mode, 0, 0, 0, 0};
    if (int rc = plan_create_on(r.M, QSIM_C64, r.ideal.data(), r.ideal.size(), &po, s->stream, &srv->alloc,
                                &s->plans[0]))
        return rc;
    if (int rc = plan_create_on(r.M, QSIM_C64, r.noisy.data(), r.noisy.size(), &po, s->stream, &srv->alloc,
                                &s->plans[1]))
        return rc;
    qsim_state st[2];
    for (int k = 0; k < 2; ++k) {
        st[k].M = r.M;
        st[k].prec = QSIM_C64;
        st[k].amps = s->amps[k];
        st[k].owned = false;
        st[k].stream = s->stream;
        st[k].scratch = s->scratch;
        st[k].scratch_blocks = kReduceSlots;
        st[k].ev = s->ev;
        st[k].alloc = srv->alloc;
        if (int rc = launch_zero_state(s->amps[k], r.M, QSIM_C64, s->stream)) return rc;
        if (int rc = qsim_plan_execute(s->plans[k], &st[k], nullptr)) return rc;
    }
    if (int rc = launch_reduce(s->amps[0], s->amps[1], r.M, QSIM_C64, s->scratch, kReduceSlots, s->stream)) return rc;
    QS_CUDA(cudaMemcpyAsync(s->h_res, s->scratch + 3 * size_t(kReduceSlots), 3 * sizeof(double),
                            cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA(cudaLaunchHostFunc(s->stream, on_slot_done, s));
    return QSIM_OK;
}

// Release the slot's resources (stream-ordered) and record the result.
void retire(qsim_server *srv, Slot *s, std::vector<qsim_request_result> &out) {
    qsim_request_result res{};
    res.id = s->req.id;
    res.M = s->req.M;
    res.n_gates = int32_t(s->req.noisy.size());
    res.status = s->status;
    if (s->status == QSIM_OK) {
        res.F = s->h_res[1] * s->h_res[1] + s->h_res[2] * s->h_res[2];
        res.norm = s->h_res[0];
        res.t_done = s->t_done.load();
    } else {
        res.t_done = srv->now();
    }
    res.t_submit = s->req.t_submit;
    res.t_start = s->t_start;
    for (int k = 0; k < 2; ++k) {
        if (s->plans[k]) plan_release(s->plans[k]);
        s->plans[k] = nullptr;
        if (s->amps[k]) {
            if (srv->alloc.free) dfree(srv->alloc, s->amps[k], (size_t(1) << s->req.M) * 8, s->stream);
            else cudaFreeAsync(s->amps[k], s->stream);
        }
        s->amps[k] = nullptr;
    }
    srv->bytes_in_use -= s->bytes;
    s->bytes = 0;
    s->busy = false;
    s->done.store(0);
    out.push_back(res);
}

void scheduler(qsim_server *srv) {
    cudaSetDevice(srv->device);
    std::vector<qsim_request_result> finished;
    std::unique_lock<std::mutex> lock(srv->mu);
    for (;;) {
        // 1. retire completed requests
        finished.clear();
        int active = 0;
        for (Slot *s : srv->slots) {
            if (s->busy && s->done.load()) retire(srv, s, finished);
            if (s->busy) ++active;
        }
        // 2. admit the oldest waiting requests while a slot and the budget allow
        while (!srv->pending.empty()) {
            Request &r = srv->pending.front();
            const size_t need = request_bytes(r.M);
            if (need > srv->opts.hbm_budget) {  // can never fit
                qsim_request_result res{};
                res.id = r.id;
                res.M = r.M;
                res.n_gates = int32_t(r.noisy.size());
                res.status = QSIM_ENOMEM;
                res.t_submit = r.t_submit;
                res.t_start = res.t_done = srv->now();
                finished.push_back(res);
                srv->pending.pop_front();
                continue;
            }
            Slot *free_slot = nullptr;
            for (Slot *s : srv->slots)
                if (!s->busy) {
                    free_slot = s;
                    break;
                }
            if (!free_slot || srv->bytes_in_use + need > srv->opts.hbm_budget) break;
            free_slot->req = std::move(r);
            srv->pending.pop_front();
            free_slot->busy = true;
            free_slot->bytes = need;
            free_slot->t_start = srv->now();
            free_slot->status = QSIM_OK;
            srv->bytes_in_use += need;
            if (srv->bytes_in_use > srv->peak_bytes) srv->peak_bytes = srv->bytes_in_use;
            ++active;
            if (active > srv->max_active) srv->max_active = active;
            lock.unlock();
            const int rc = start_request(srv, free_slot);
            lock.lock();
            if (rc != QSIM_OK) {  // fail this request once its queued work (if any) has drained
                free_slot->status = rc;
                lock.unlock();
                cudaStreamSynchronize(free_slot->stream);
                cudaGetLastError();
                lock.lock();
                retire(srv, free_slot, finished);
                --active;
            }
        }
        if (!finished.empty()) {
            for (auto &res : finished) srv->done.push_back(res);
            srv->n_completed += finished.size();
            srv->cv_done.notify_all();
        }
        if (srv->stop && srv->pending.empty() && active == 0) break;
        bool ready = false;
        for (Slot *s : srv->slots) ready |= s->busy && s->done.load();
        if (!ready) srv->cv_work.wait_for(lock, std::chrono::milliseconds(5));
    }
}

}  // namespace

extern "C" {

int qsim_server_create(const qsim_server_opts *opts, qsim_server **out) {
    if (!opts || !out) { set_error("opts or out is NULL"); return QSIM_EINVAL; }
    if (opts->max_slots < 1 || opts->max_slots > 256) {
        set_error("max_slots %d outside [1, 256]", opts->max_slots);
        return QSIM_EINVAL;
    }
    if (opts->hbm_budget == 0) { set_error("hbm_budget is 0"); return QSIM_EINVAL; }
    if (opts->mode < QSIM_MODE_AUTO || opts->mode > QSIM_MODE_FUSED) { set_error("unknown mode"); return QSIM_EINVAL; }
    qsim_server *srv = new qsim_server();
    srv->opts = *opts;
    srv->t0 = Clock::now();
    auto fail = [&](int rc) {
        qsim_server_destroy(srv);
        return rc;
    };
    if (cudaGetDevice(&srv->device) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "cudaGetDevice"));
    srv->alloc = current_allocator();
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = srv->device;
    if (cudaError_t e = cudaMemPoolCreate(&srv->pool, &props)) return fail(cuda_fail(e, "memory pool"));
    uint64_t keep = opts->hbm_budget;
    cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    for (int i = 0; i < opts->max_slots; ++i) {
        Slot *s = new Slot();
        s->srv = srv;
        srv->slots.push_back(s);
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_res, 4 * sizeof(double));
        if (e != cudaSuccess) return fail(cuda_fail(e, "server slot"));
        if (int rc = dmalloc(srv->alloc, reinterpret_cast<void **>(&s->scratch), state_scratch_bytes(kReduceSlots),
                             nullptr, "server slot scratch"))
            return fail(rc);
    }
    if (int rc = tile_prepare(QSIM_C64)) return fail(rc);
    if (int rc = fused_prepare()) return fail(rc);
    srv->worker = std::thread(scheduler, srv);
    *out = srv;
    return QSIM_OK;
}

int qsim_server_submit(qsim_server *srv, int M, const qsim_gate *ideal, const qsim_gate *noisy, size_t n,
                       uint64_t *id) {
    if (!srv) { set_error("server is NULL"); return QSIM_EINVAL; }
    if (M < 1 || M > QSIM_MAX_QUBITS) { set_error("M = %d outside [1, %d]", M, QSIM_MAX_QUBITS); return QSIM_EINVAL; }
    if (n > 0 && (!ideal || !noisy)) { set_error("gates are NULL"); return QSIM_EINVAL; }
    for (size_t i = 0; i < n; ++i) {
        Gate g;
        for (const qsim_gate *x : {ideal + i, noisy + i})
            if (int rc = make_gate(M, x->U, x->target, x->controls, x->ncontrols, &g)) return rc;
    }
    Request r;
    r.M = M;
    r.ideal.assign(ideal, ideal + n);
    r.noisy.assign(noisy, noisy + n);
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->stop) { set_error("server is shutting down"); return QSIM_EINVAL; }
    if (srv->pending.size() >= kMaxPending) { set_error("request queue full"); return QSIM_EBUSY; }
    r.id = srv->next_id++;
    r.t_submit = srv->now();
    if (id) *id = r.id;
    srv->pending.push_back(std::move(r));
    ++srv->n_submitted;
    srv->cv_work.notify_all();
    return QSIM_OK;
}

int qsim_server_poll(qsim_server *srv, qsim_request_result *out, int max, int *nout, int wait_ms) {
    if (!srv || !nout || (max > 0 && !out)) { set_error("bad arguments"); return QSIM_EINVAL; }
    std::unique_lock<std::mutex> lock(srv->mu);
    if (srv->done.empty() && wait_ms > 0)
        srv->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return !srv->done.empty(); });
    int k = 0;
    while (k < max && !srv->done.empty()) {
        out[k++] = srv->done.front();
        srv->done.pop_front();
    }
    *nout = k;
    return QSIM_OK;
}

int qsim_server_get_stats(qsim_server *srv, qsim_server_stats *out) {
    if (!srv || !out) { set_error("bad arguments"); return QSIM_EINVAL; }
    std::lock_guard<std::mutex> lock(srv->mu);
    out->n_submitted = srv->n_submitted;
    out->n_completed = srv->n_completed;
    out->n_pending = srv->pending.size();
    out->bytes_in_use = srv->bytes_in_use;
    out->peak_bytes = srv->peak_bytes;
    out->max_active = srv->max_active;
    out->now = srv->now();
    return QSIM_OK;
}

void qsim_server_destroy(qsim_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    for (Slot *s : srv->slots) {
        if (s->stream) cudaStreamSynchronize(s->stream);
        dfree(srv->alloc, s->scratch, state_scratch_bytes(kReduceSlots), nullptr);
        if (s->h_res) cudaFreeHost(s->h_res);
        if (s->ev) cudaEventDestroy(s->ev);
        if (s->stream) cudaStreamDestroy(s->stream);
        delete s;
    }
    if (srv->pool) cudaMemPoolDestroy(srv->pool);
    delete srv;
}

}  // extern "C"
