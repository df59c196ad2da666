// ms_cvae_train_step_static: one CVAE training step whose scratch memory is a fixed array inside this
// library, so the caller passes no workspace and nothing is allocated.
//
// Who needs it: code that may not call cudaMalloc (or any allocating routine) at the point where it trains
// — for example a host whose device memory is entirely owned by another framework's pool, or a plug-in that
// must not allocate while the application runs.  Such a caller passes only its parameters, optimiser state,
// batch and loss buffers, as for ms_cvae_train_step.
//
// The scratch (per-block gradient partials and the reduced gradient, ms_cvae_workspace_size bytes) lives
// in the file-scope array below.  Every device that loads the library holds kStaticScratchBytes for it until
// the process exits.  All calls share it: two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it and corrupt each other's gradient.  Each call overwrites everything it
// reads (partials are written in full before the reduction, the gradient before Adam), so nothing in the
// array has to be cleared between calls.
//
// In host code the array's name is only a stand-in for its device address, so the address is looked up once
// per device with cudaGetSymbolAddress, with that device current, on the first call made on it; make that
// first call before any stream capture.
#include <mutex>

#include "ms_device.cuh"

namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_train_scratch[kStaticScratchBytes];

std::mutex g_lock;
void* g_scratch_addr[kMaxDevices] = {};

cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_train_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" size_t ms_cvae_static_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" ms_status ms_cvae_train_step_static(const ms_cvae_shape* s, float* params, float* m, float* v,
                                               const float* x, const float* c, const float* eps_z, uint64_t B,
                                               uint64_t seed, uint64_t step, float lr, float weight_decay,
                                               float* loss3, void* stream)
{
    MS_CHECK_ARG(s != nullptr, "ms_cvae_train_step_static: null shape");
    const size_t need = ms_cvae_workspace_size(s, B);
    MS_CHECK_ARG(need <= kStaticScratchBytes,
                 "ms_cvae_train_step_static: batch %llu needs %zu bytes of scratch, more than the %zu-byte static "
                 "array; use ms_cvae_train_step with a workspace, or a smaller batch",
                 (unsigned long long)B, need, kStaticScratchBytes);
    void* scratch = nullptr;
    MS_CUDA(scratch_address(&scratch));
    return ms_cvae_train_step(s, params, m, v, x, c, eps_z, B, seed, step, lr, weight_decay, loss3, scratch,
                              kStaticScratchBytes, stream);
}
