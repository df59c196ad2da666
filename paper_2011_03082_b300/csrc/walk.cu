// ms_simulate_walks: argument validation and launch of the persistent walk (walk_impl.cuh).
#include <cmath>

#include "walk_impl.cuh"

namespace ms {
namespace walk {
cudaError_t launch_f64(const Job& J, cudaStream_t stream);
}  // namespace walk
}  // namespace ms

extern "C" size_t ms_walk_workspace_size(const ms_walk_params* p)
{
    (void)p;
    return 256;
}

extern "C" ms_status ms_simulate_walks(const ms_walk_params* p, const ms_walk_out* out, void* workspace,
                                       size_t workspace_bytes, void* stream)
{
    MS_NVTX("ms_simulate_walks");
    MS_CHECK_ARG(p != nullptr && out != nullptr, "ms_simulate_walks: null params or outputs");
    MS_CHECK_ARG(p->media != nullptr, "ms_simulate_walks: media is null");
    MS_CHECK_ARG(p->max_events >= 1, "ms_simulate_walks: max_events must be >= 1");
    MS_CHECK_ARG(p->reservoir >= 0 && p->reservoir <= 2, "ms_simulate_walks: reservoir must be 0, 1 or 2");
    MS_CHECK_ARG(p->precision == MS_FP32 || p->precision == MS_FP64,
                 "ms_simulate_walks: precision must be MS_FP32 or MS_FP64");
    MS_CHECK_ARG(p->n_photons < (1ull << 62), "ms_simulate_walks: n_photons too large");
    MS_CHECK_ARG(workspace != nullptr && workspace_bytes >= ms_walk_workspace_size(p),
                 "ms_simulate_walks: workspace of at least %zu bytes required", ms_walk_workspace_size(p));
    MS_CHECK_ARG(((uintptr_t)workspace & 255u) == 0, "ms_simulate_walks: workspace must be 256-byte aligned");
    if (p->n_photons == 0) return MS_OK;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p->media) != cudaSuccess || (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return ms::set_error(MS_ERR_INVALID_ARG, "ms_simulate_walks: media must be a device pointer");
    }
    ms::walk::Job J;
    J.seed = p->seed;
    J.offset = p->photon_offset;
    J.n = p->n_photons;
    J.media = p->media;
    J.per_photon_media = p->per_photon_media;
    J.max_events = p->max_events;
    J.reservoir = p->reservoir;
    J.out = *out;
    J.ticket = static_cast<unsigned long long*>(workspace);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MS_CUDA(cudaMemsetAsync(workspace, 0, sizeof(unsigned long long), s));
    if (p->precision == MS_FP64) {
        MS_CUDA(ms::walk::launch_f64(J, s));
    } else {
        MS_CUDA((ms::walk::launch<ms::walk::F32>(J, s)));
    }
    return MS_OK;
}
