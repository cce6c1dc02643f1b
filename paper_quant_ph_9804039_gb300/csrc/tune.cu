// Measured autotuning.  The execution forms of a circuit (tile passes of
// 2^11 or 2^12 amplitudes, fused tensor-core blocks of k = 3, 4 or 5 qubits)
// are chosen by a time model of the planned passes whose rates are measured
// on the device: the bandwidth of a light tile pass, the FMA rate of a heavy
// one, the bandwidth of the permutation pass, and of a fused block of each
// width on and off qubits 0..4.  The rates are measured once per device,
// precision and kernel kind (general or specialised tile passes) on a
// 26-qubit state (512 MiB for complex64, larger than L2) filled with dense
// pseudo-random amplitudes (a state of zeros runs the same launches faster:
// at M=33, 6.18 against 6.04 TB/s for a fused block with direct stores and
// 5.49 against 4.66 TB/s for a staged one), and kept in memory
// and in a JSON cache file (qsim_tune_set_cache), so that later processes
// replay them.  The trajectory plans keep their timed configuration in the
// same file.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <ctime>
#include <map>
#include <mutex>
#include <string>

#include "qsim_internal.h"

namespace qs {

namespace {

// Dense amplitudes of modulus ~2^(-M/2): a 32-bit integer hash of the index
// gives each real and imaginary part a value in [-1, 1), scaled.
template <typename R>
__global__ void k_fill_dense(R *re_im, uint64_t n_reals, R scale) {
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n_reals;
         i += uint64_t(gridDim.x) * blockDim.x) {
        uint32_t h = uint32_t(i) * 0x9E3779B1u ^ uint32_t(i >> 32) * 0x85EBCA77u;
        h ^= h >> 15;
        h *= 0x2C1B3C6Du;
        h ^= h >> 12;
        h *= 0x297A2D39u;
        h ^= h >> 15;
        re_im[i] = scale * (R(int32_t(h)) * R(1.0 / 2147483648.0));
    }
}

std::mutex g_mu;
bool g_path_set = false;
std::string g_path;  // "" = memory only
std::map<std::string, std::map<std::string, double>> g_store;
bool g_loaded = false;

const std::string &cache_path() {
    if (!g_path_set) {
        const char *env = std::getenv("QSIM_TUNE_CACHE");
        g_path = env ? env : "";
        g_path_set = true;
    }
    return g_path;
}

// The file: one JSON object, one entry per line, "key": {"name": number, ...}.
void load_file() {
    if (g_loaded) return;
    g_loaded = true;
    const std::string &path = cache_path();
    if (path.empty()) return;
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return;
    char line[4096];
    while (std::fgets(line, sizeof line, f)) {
        const char *p = std::strchr(line, '"');
        if (!p) continue;
        const char *q = std::strchr(p + 1, '"');
        if (!q) continue;
        const std::string key(p + 1, q);
        const char *b = std::strchr(q, '{');
        if (!b) continue;
        std::map<std::string, double> vals;
        const char *c = b + 1;
        for (;;) {
            const char *n0 = std::strchr(c, '"');
            if (!n0) break;
            const char *n1 = std::strchr(n0 + 1, '"');
            if (!n1) break;
            const char *colon = std::strchr(n1, ':');
            if (!colon) break;
            char *end = nullptr;
            const double v = std::strtod(colon + 1, &end);
            if (end == colon + 1) break;
            vals[std::string(n0 + 1, n1)] = v;
            c = end;
        }
        if (!vals.empty() && !g_store.count(key)) g_store[key] = vals;
    }
    std::fclose(f);
}

void save_file() {
    const std::string &path = cache_path();
    if (path.empty()) return;
    const std::string tmp = path + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n");
    size_t i = 0;
    for (const auto &kv : g_store) {
        std::fprintf(f, "\"%s\": {", kv.first.c_str());
        size_t j = 0;
        for (const auto &nv : kv.second)
            std::fprintf(f, "\"%s\": %.9g%s", nv.first.c_str(), nv.second, ++j < kv.second.size() ? ", " : "");
        std::fprintf(f, "}%s\n", ++i < g_store.size() ? "," : "");
    }
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path.c_str());
}

std::string device_name() {
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    char buf[320];
    std::snprintf(buf, sizeof buf, "%s sm_%d%d", prop.name, prop.major, prop.minor);
    return buf;
}

// Milliseconds of one execution of the plan on st (in place), the median of
// three after one untimed run.
int time_plan(qsim_plan *plan, qsim_state *st, double *ms) {
    cudaEvent_t e[4];
    for (cudaEvent_t &x : e) QS_CUDA(cudaEventCreate(&x));
    int rc = qsim_plan_execute(plan, st, nullptr);
    float t[3] = {0, 0, 0};
    for (int r = 0; r < 3 && rc == QSIM_OK; ++r) {
        cudaEventRecord(e[0], st->stream);
        rc = qsim_plan_execute(plan, st, nullptr);
        cudaEventRecord(e[1], st->stream);
        if (rc == QSIM_OK) {
            cudaError_t err = cudaEventSynchronize(e[1]);
            if (err != cudaSuccess) rc = cuda_fail(err, "tuning run");
            else cudaEventElapsedTime(&t[r], e[0], e[1]);
        }
    }
    for (cudaEvent_t &x : e) cudaEventDestroy(x);
    std::sort(t, t + 3);
    *ms = t[1];
    return rc;
}

qsim_gate rec(const double *U, int t, int nc = 0, int c0 = 0, int c1 = 0) {
    qsim_gate g{};
    std::memcpy(g.U, U, sizeof g.U);
    g.target = t;
    g.ncontrols = nc;
    g.controls[0] = c0;
    g.controls[1] = c1;
    return g;
}

// A fixed dense unitary (a rotation with a phase), different per index.
void dense_u(int i, double *U) {
    const double a = 0.37 + 0.11 * i, b = 1.3 - 0.07 * i, c = 0.5 + 0.05 * i;
    const double ca = std::cos(a), sa = std::sin(a);
    // [[ca e^{ib}, -sa e^{-ic}], [sa e^{ic}, ca e^{-ib}]]
    U[0] = ca * std::cos(b); U[1] = ca * std::sin(b);
    U[2] = -sa * std::cos(c); U[3] = sa * std::sin(c);
    U[4] = sa * std::cos(c); U[5] = sa * std::sin(c);
    U[6] = ca * std::cos(b); U[7] = -ca * std::sin(b);
}

constexpr int kTuneM = 26;

int measure(qsim_prec prec, bool spec, std::map<std::string, double> &v) {
    const int M = kTuneM;
    const double N = std::ldexp(1.0, M), ab = double(amp_bytes(prec));
    qsim_state *st = nullptr;
    if (int rc = qsim_alloc(M, prec, &st)) return rc;
    int rc = QSIM_OK;
    {
        const uint64_t n_reals = uint64_t(2) << M;
        if (prec == QSIM_C64)
            k_fill_dense<float><<<4 * num_sms(), 256, 0, st->stream>>>(static_cast<float *>(st->amps), n_reals,
                                                                        float(std::ldexp(1.0, -M / 2)));
        else
            k_fill_dense<double><<<4 * num_sms(), 256, 0, st->stream>>>(static_cast<double *>(st->amps), n_reals,
                                                                         std::ldexp(1.0, -M / 2));
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
        if (e != cudaSuccess) {
            qsim_free(st);
            return cuda_fail(e, "filling the tuning state");
        }
    }
    auto run = [&](const std::vector<qsim_gate> &g, int mode, int tile_bits, int fuse_k, double *ms,
                   double *fma_amp) -> int {
        qsim_opts o{};
        o.mode = mode;
        o.tile_bits = tile_bits;
        o.fuse_k = fuse_k;
        o.specialize = spec ? 1 : 0;
        qsim_plan *pl = nullptr;
        if (int r = qsim_plan_create(M, prec, g.data(), g.size(), &o, &pl)) return r;
        if (fma_amp) *fma_amp = plan_model_fma(pl);
        int r = time_plan(pl, st, ms);
        qsim_plan_destroy(pl);
        return r;
    };
    const double H[8] = {M_SQRT1_2, 0, M_SQRT1_2, 0, M_SQRT1_2, 0, -M_SQRT1_2, 0};
    const double X[8] = {0, 0, 1, 0, 1, 0, 0, 0};
    const int b = prec == QSIM_C64 ? 12 : 11;
    double ms = 0;
    {  // light tile pass: Hadamards on the tile's qubits (bandwidth)
        std::vector<qsim_gate> g;
        for (int q = 0; q < b; ++q) g.push_back(rec(H, q));
        if ((rc = run(g, QSIM_MODE_TILED, b, 0, &ms, nullptr))) goto done;
        v["pass_bw"] = 2.0 * N * ab / (ms * 1e-3);
    }
    {  // heavy tile pass: four dense complex gates per tile qubit (FMA rate)
        std::vector<qsim_gate> g;
        double U[8], fma = 0;
        for (int r = 0; r < 4; ++r)
            for (int q = 0; q < b; ++q) {
                dense_u(r * b + q, U);
                g.push_back(rec(U, q));
            }
        if ((rc = run(g, QSIM_MODE_TILED, b, 0, &ms, &fma))) goto done;
        v["fma_rate"] = fma * N / (ms * 1e-3);
    }
    {  // permutation pass: swaps of qubit pairs (0,20), (1,21), (2,22), three CNOTs each
        std::vector<qsim_gate> g;
        for (int q = 0; q < 3; ++q) {
            g.push_back(rec(X, q + 20, 1, q));
            g.push_back(rec(X, q, 1, q + 20));
            g.push_back(rec(X, q + 20, 1, q));
        }
        if ((rc = run(g, QSIM_MODE_TILED, b, 0, &ms, nullptr))) goto done;
        v["perm_bw"] = 2.0 * N * ab / (ms * 1e-3);
    }
    if (prec == QSIM_C64) {
        for (int k = 3; k <= 5; ++k) {  // one block on qubits 20.. (direct stores) and on 0.. (staged)
            for (int low = 0; low < 2; ++low) {
                std::vector<qsim_gate> g;
                double U[8];
                for (int r = 0; r < 2; ++r)
                    for (int j = 0; j < k; ++j) {
                        dense_u(r * k + j, U);
                        g.push_back(rec(U, (low ? 0 : 20) + j));
                    }
                if ((rc = run(g, QSIM_MODE_FUSED, 0, k, &ms, nullptr))) goto done;
                char name[32];
                std::snprintf(name, sizeof name, "fused%d_%s", k, low ? "staged" : "direct");
                v[name] = 2.0 * N * ab / (ms * 1e-3);
            }
        }
    }
done:
    qsim_free(st);
    return rc;
}

}  // namespace

int model_rates(qsim_prec prec, bool spec, ModelRates *r, std::string *src) {
    std::lock_guard<std::mutex> lock(g_mu);
    load_file();
    const std::string key = "rates|dense|" + device_name() + "|" + (prec == QSIM_C64 ? "c64" : "c128") + "|" +
                            (spec ? "specialised" : "general");
    auto it = g_store.find(key);
    bool measured_now = false;
    if (it == g_store.end()) {
        std::map<std::string, double> v;
        if (int rc = measure(prec, spec, v)) return rc;
        v["M"] = kTuneM;
        v["unix_time"] = double(std::time(nullptr));
        g_store[key] = v;
        save_file();
        it = g_store.find(key);
        measured_now = true;
    }
    const std::map<std::string, double> &v = it->second;
    auto get = [&](const char *n, double dflt) {
        auto j = v.find(n);
        return j != v.end() && j->second > 0 ? j->second : dflt;
    };
    r->pass_bw = get("pass_bw", 6.0e12);
    r->fma_rate = get("fma_rate", 2.2e13);
    r->perm_bw = get("perm_bw", 3.6e12);
    for (int k = 0; k < 6; ++k) {
        char a[32], b[32];
        std::snprintf(a, sizeof a, "fused%d_direct", k);
        std::snprintf(b, sizeof b, "fused%d_staged", k);
        r->fused_direct[k] = get(a, 5.0e12);
        r->fused_staged[k] = get(b, 4.5e12);
    }
    if (src)
        *src = (measured_now ? "measured now (" : "replayed from the cache (") + key + ")";
    return QSIM_OK;
}

int tune_lookup(const std::string &key, double *value) {
    std::lock_guard<std::mutex> lock(g_mu);
    load_file();
    auto it = g_store.find(key);
    if (it == g_store.end()) return 0;
    auto j = it->second.find("value");
    if (j == it->second.end()) return 0;
    *value = j->second;
    return 1;
}

void tune_record(const std::string &key, double value) {
    std::lock_guard<std::mutex> lock(g_mu);
    load_file();
    g_store[key] = {{"value", value}, {"unix_time", double(std::time(nullptr))}};
    save_file();
}

std::string tune_device_key() { return device_name(); }

}  // namespace qs

extern "C" int qsim_tune_set_cache(const char *path) {
    std::lock_guard<std::mutex> lock(qs::g_mu);
    qs::g_path = path ? path : "";
    qs::g_path_set = true;
    qs::g_loaded = false;
    qs::g_store.clear();
    return QSIM_OK;
}

extern "C" int qsim_tune_rates(int prec, int specialize, char *buf, int64_t len, int64_t *needed) {
    if (prec != QSIM_C64 && prec != QSIM_C128) {
        qs::set_error("unknown precision %d", prec);
        return QSIM_EINVAL;
    }
    qs::ModelRates r{};
    std::string src;
    if (int rc = qs::model_rates(qsim_prec(prec), specialize != 0, &r, &src)) return rc;
    char text[1024];
    std::snprintf(text, sizeof text,
                  "{\"source\": \"%s\", \"pass_bw\": %.6g, \"fma_rate\": %.6g, \"perm_bw\": %.6g, "
                  "\"fused_direct\": [%.6g, %.6g, %.6g], \"fused_staged\": [%.6g, %.6g, %.6g]}",
                  src.c_str(), r.pass_bw, r.fma_rate, r.perm_bw, r.fused_direct[3], r.fused_direct[4],
                  r.fused_direct[5], r.fused_staged[3], r.fused_staged[4], r.fused_staged[5]);
    const std::string out = text;
    if (needed) *needed = int64_t(out.size()) + 1;
    if (len > 0 && buf) {
        const size_t n = std::min(out.size(), size_t(len - 1));
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return QSIM_OK;
}
