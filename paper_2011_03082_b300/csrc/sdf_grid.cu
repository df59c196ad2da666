// ms_sdf_grid_build: the voxel grid of conservative distances to the object's surface that sizes the sphere
// steps (Sec. 3: the bounding volume is voxelised in a pre-process and each voxel holds a conservative
// shortest distance to the surface).  The object is the displaced unit sphere f(p) = |p| - 1 - A s(p),
// s(p) = sin(kx) sin(ky) sin(kz), whose Lipschitz constant is 1 + A k.
//
// 1. A voxel may hold surface only if |f(c)| <= (1 + A k) h sqrt(3) / 2 at its centre c (f cannot change sign
//    closer to c than |f(c)| / (1 + A k), and no point of the voxel is farther than h sqrt(3) / 2 from c).
// 2. The exact Euclidean distance transform of those voxels over the grid, in voxel units, as three separable
//    passes (x, then y, then z): each voxel takes the minimum over its line of (the previous pass's squared
//    distance + the squared index offset); integers throughout, so the result does not depend on scheduling.
// 3. The value is (e - sqrt(3)) h, clamped at 0, with e the distance between the voxel's centre and the
//    nearest such voxel's centre: two points of two voxels are at most a diagonal, sqrt(3) h, nearer than
//    their centres.  (The paper stores a Chebyshev distance; the Euclidean one is also conservative and up to
//    sqrt(3) times larger along diagonals, hence larger spheres.)
#include "ms_device.cuh"

namespace ms {
namespace grid {

constexpr int kFar = 1 << 28;   // "no voxel that may hold surface on this line"; sums of three stay below 2^31

__global__ void mark_kernel(float A, float k, int n, float b, float h, int* __restrict__ m)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n * n) return;
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((int64_t)n * n));
    const float cx = -b + (ix + 0.5f) * h, cy = -b + (iy + 0.5f) * h, cz = -b + (iz + 0.5f) * h;
    const float f = sqrtf(cx * cx + cy * cy + cz * cz) - 1.0f - A * sinf(k * cx) * sinf(k * cy) * sinf(k * cz);
    m[i] = fabsf(f) <= (1.0f + A * k) * 0.8660254037844386f * h ? 0 : kFar;
}

// One separable pass along axis `axis` (0 = x, 1 = y, 2 = z): dst(v) = min over the line through v of
// src(w) + (index offset)^2, with src values kFar meaning "none" (they stay kFar unless a real value wins).
__global__ void edt_pass_kernel(int n, int axis, const int* __restrict__ src, int* __restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n * n) return;
    const int c[3] = {(int)(i % n), (int)((i / n) % n), (int)(i / ((int64_t)n * n))};
    const int64_t stride = axis == 0 ? 1 : (axis == 1 ? n : (int64_t)n * n);
    const int64_t base = i - (int64_t)c[axis] * stride;
    int best = kFar;
    for (int j = 0; j < n; ++j) {
        const int v = src[base + (int64_t)j * stride];
        if (v >= kFar) continue;
        const int d = j - c[axis];
        best = min(best, v + d * d);
    }
    dst[i] = best;
}

__global__ void value_kernel(int n, float h, const int* __restrict__ e2, float* __restrict__ g)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n * n) return;
    const float e = e2[i] >= kFar ? 3.0e4f : sqrtf((float)e2[i]);
    g[i] = fmaxf(0.0f, (e - 1.7320508075688772f) * h);
}

}  // namespace grid
}  // namespace ms

extern "C" size_t ms_sdf_grid_workspace_size(int32_t n)
{
    return n < 1 ? 0 : (size_t)2 * n * n * n * sizeof(int);
}

extern "C" ms_status ms_sdf_grid_build(float disp_amp, float disp_freq, int32_t n, float* grid, void* workspace,
                                       size_t workspace_bytes, void* stream)
{
    MS_NVTX("ms_sdf_grid_build");
    MS_CHECK_ARG(grid != nullptr, "ms_sdf_grid_build: null grid");
    MS_CHECK_ARG(n >= 4 && n <= 1024, "ms_sdf_grid_build: n must be in 4..1024");
    MS_CHECK_ARG(disp_amp >= 0.0f && disp_amp < 1.0f && disp_freq >= 0.0f,
                 "ms_sdf_grid_build: need 0 <= disp_amp < 1 and disp_freq >= 0");
    MS_CHECK_ARG(workspace != nullptr && workspace_bytes >= ms_sdf_grid_workspace_size(n) &&
                     ((uintptr_t)workspace & 15u) == 0,
                 "ms_sdf_grid_build: a 16-byte aligned workspace of ms_sdf_grid_workspace_size(n) bytes is required");
    const float h = 2.0f * (1.0f + disp_amp) / (float)(n - 2), b = 1.0f + disp_amp + h;
    const int64_t total = (int64_t)n * n * n;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* a = static_cast<int*>(workspace);
    int* c = a + total;
    ms::grid::mark_kernel<<<blocks, 256, 0, s>>>(disp_amp, disp_freq, n, b, h, a);
    ms::grid::edt_pass_kernel<<<blocks, 256, 0, s>>>(n, 0, a, c);
    ms::grid::edt_pass_kernel<<<blocks, 256, 0, s>>>(n, 1, c, a);
    ms::grid::edt_pass_kernel<<<blocks, 256, 0, s>>>(n, 2, a, c);
    ms::grid::value_kernel<<<blocks, 256, 0, s>>>(n, h, c, grid);
    MS_CUDA(cudaGetLastError());
    return MS_OK;
}
