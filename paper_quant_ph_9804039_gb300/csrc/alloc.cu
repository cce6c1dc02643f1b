// Device memory of the library.  Every device allocation the library makes
// (state amplitudes and reduction scratch, plan tables, trajectory workspaces,
// the server's state vectors) goes through one function pair: the caller's
// hook when one is set with qsim_set_allocator (for instance a framework's
// caching allocator, so that the library shares its pool), else the CUDA
// runtime.  Each object keeps the pair it was created with and releases its
// memory through it.
#include <mutex>

#include "qsim_internal.h"

namespace qs {

namespace {
std::mutex g_alloc_mu;
DevAllocator g_alloc{nullptr, nullptr, nullptr};
}  // namespace

DevAllocator current_allocator() {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    return g_alloc;
}

int dmalloc(const DevAllocator &a, void **p, size_t bytes, cudaStream_t s, const char *what) {
    *p = nullptr;
    if (bytes == 0) return QSIM_OK;
    if (a.alloc) {
        *p = a.alloc(bytes, s, a.ctx);
        if (!*p) {
            set_error("the allocator hook returned NULL for %zu bytes (%s)", bytes, what);
            return QSIM_ENOMEM;
        }
        if (reinterpret_cast<uintptr_t>(*p) & 255) {
            a.free(*p, bytes, s, a.ctx);
            *p = nullptr;
            set_error("the allocator hook returned memory that is not 256-byte aligned (%s)", what);
            return QSIM_EINVAL;
        }
        return QSIM_OK;
    }
    cudaError_t e = s ? cudaMallocAsync(p, bytes, s) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cannot allocate %zu bytes of device memory (%s): %s", bytes, what, cudaGetErrorString(e));
        return QSIM_ENOMEM;
    }
    return QSIM_OK;
}

void dfree(const DevAllocator &a, void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (a.free) {
        a.free(p, bytes, s, a.ctx);
        return;
    }
    if (s) cudaFreeAsync(p, s);
    else cudaFree(p);
}

}  // namespace qs

extern "C" int qsim_set_allocator(qsim_device_alloc_fn alloc, qsim_device_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        qs::set_error("qsim_set_allocator: give both functions or neither");
        return QSIM_EINVAL;
    }
    std::lock_guard<std::mutex> lock(qs::g_alloc_mu);
    qs::g_alloc = qs::DevAllocator{alloc, free_fn, alloc ? ctx : nullptr};
    return QSIM_OK;
}
