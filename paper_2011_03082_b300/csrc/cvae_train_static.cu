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
// In host code the array's name is only a stand-in for its device address, so the address is looked up with
// cudaGetSymbolAddress, with the device current, on the first call made on a device, and kept together with
// the identity of the CUDA context it belongs to.  A later call in another context of that device (after
// cudaDeviceReset, which destroys the primary context and with it the module's memory) looks it up again.
// Context identities come from cuCtxGetId, which never reuses an identity within a process (the driver
// functions are reached through cudaGetDriverEntryPointByVersion, so the library does not link libcuda).
// Make the first call on a device, and the first one after a reset, before any stream capture.
#include <cuda.h>   // driver API types only

#include <mutex>

#include "ms_device.cuh"

namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_train_scratch[kStaticScratchBytes];

struct Resolved {
    unsigned long long ctx_id;   // cuCtxGetId of the context the address belongs to (0: none yet)
    void* addr;
};

std::mutex g_lock;
Resolved g_scratch[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Identity of the calling thread's current context, or 0 when there is none (or the driver cannot say).
unsigned long long current_context_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    Resolved& r = g_scratch[dev];
    const unsigned long long id = current_context_id();
    if (r.addr == nullptr || id == 0 || id != r.ctx_id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_train_scratch);   // creates the device's primary context if needed
        if (e != cudaSuccess) return e;
        r.addr = p;
        r.ctx_id = current_context_id();
    }
    *out = r.addr;
    return cudaSuccess;
}

}  // namespace

extern "C" size_t ms_cvae_static_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" ms_status ms_cvae_train_step_static(const ms_cvae_shape* s, float* params, float* m, float* v,
                                               const float* x, const float* c, const float* eps_z, uint64_t B,
                                               uint64_t seed, uint64_t step, float lr, float weight_decay,
                                               float* loss3, void* stream)
{
    MS_NVTX("ms_cvae_train_step_static");
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
