// ms_cvae_infer: batched CVAE decoder sampling (Sec. 3.2) — x = mu + exp(log Sigma / 2) eps with
// (mu, log Sigma) = Dec([c; z]) and z, eps standard normal.
//
// Every precision runs on the tensor cores (mma.sync m16n8k16, FP32 accumulation; decoder_mma.cuh), 32 queries
// per warp over a grid-stride loop; the block stages the decoder weights once in shared memory in fragment
// order; z and eps are read from the caller or drawn from the query's Philox counter.
//   MS_FP32: weights and activations split into FP16 head + tail, three products per tile (about 22
//            significant bits: single-precision results, max |error| <= 1e-5 on the outputs);
//   MS_FP16 / MS_BF16: weights rounded once to half precision, activations split into head + tail (two
//            products per tile), so the result is that of the rounded weights.
#include "decoder.cuh"
#include "decoder_mma.cuh"

namespace ms {
namespace dec {

// Runtime-shaped kernel (any supported shape): rows are staged through shared memory.
constexpr int kMmaThreads = 128;

template <int NT3, int NTH, bool kBF16, int kSplit>
__global__ void __launch_bounds__(kMmaThreads) infer_mma(const float* __restrict__ wts, int p_in, int latent, int p_out,
                                                         const float* __restrict__ cond, const float* __restrict__ z_eps,
                                                         uint64_t seed, uint64_t offset, uint64_t n,
                                                         float* __restrict__ mlv, float* __restrict__ smp)
{
    __shared__ __align__(16) unsigned char wsm[mmadec::smem_bytes(8, NTH)];
    __shared__ float stage[kMmaThreads / 32][mmadec::kStageFloats];
    __shared__ float rows[kMmaThreads][41];   // [0,16) inputs, [16,24) eps, [24,40) outputs
    mmadec::stage_weights<kBF16, NTH, kSplit == 3>(wsm, wts, p_in + latent, p_out);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* my = rows[threadIdx.x];
    const int nz = latent + p_out;
    const uint64_t n_chunks = (n + 31) / 32;
    const uint64_t warps = (uint64_t)gridDim.x * (kMmaThreads / 32);
    for (uint64_t ch = (uint64_t)blockIdx.x * (kMmaThreads / 32) + warp; ch < n_chunks; ch += warps) {
        const uint64_t q = ch * 32 + lane;
        const bool live = q < n;
        for (int k = 0; k < 24; ++k) my[k] = 0.0f;
        if (live) {
            for (int k = 0; k < p_in; ++k) my[k] = cond[q * p_in + k];
            if (z_eps) {
                for (int m = 0; m < nz; ++m) my[m < latent ? p_in + m : 16 + m - latent] = z_eps[q * nz + m];
            } else {
                float v[16];
                query_normals_runtime(Stream(seed, offset + q), 0xD0u, nz, v);
                for (int m = 0; m < nz; ++m) my[m < latent ? p_in + m : 16 + m - latent] = v[m];
            }
        }
        float x[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = my[k];
        float y[8 * NT3];
        mmadec::warp_mlp<NT3, kSplit, kBF16, NTH>(wsm, stage[warp], x, y);
        if (live) {
#pragma unroll
            for (int j = 0; j < 8 * NT3; ++j) my[24 + j] = y[j];
            if (mlv)
                for (int o = 0; o < 2 * p_out; ++o) mlv[q * (2 * p_out) + o] = my[24 + o];
            if (smp)
                for (int o = 0; o < p_out; ++o)
                    smp[q * p_out + o] = my[24 + o] + __expf(0.5f * my[24 + p_out + o]) * my[16 + o];
        }
    }
}

cudaError_t launch_infer_mma(const ms_decoder& d, const float* cond, const float* z_eps, uint64_t seed, uint64_t offset,
                             uint64_t n, float* mlv, float* smp, cudaStream_t stream)
{
    const bool w8 = d.width == 8, one = mmadec::n_tiles_out(d.p_out) == 1;
    auto kern = d.precision == MS_BF16
                    ? (one ? (w8 ? infer_mma<1, 1, true, 2> : infer_mma<1, 2, true, 2>)
                           : (w8 ? infer_mma<2, 1, true, 2> : infer_mma<2, 2, true, 2>))
                : d.precision == MS_FP16
                    ? (one ? (w8 ? infer_mma<1, 1, false, 2> : infer_mma<1, 2, false, 2>)
                           : (w8 ? infer_mma<2, 1, false, 2> : infer_mma<2, 2, false, 2>))
                    : (one ? (w8 ? infer_mma<1, 1, false, 3> : infer_mma<1, 2, false, 3>)
                           : (w8 ? infer_mma<2, 1, false, 3> : infer_mma<2, 2, false, 3>));
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMmaThreads, 0);
    if (e != cudaSuccess) return e;
    uint64_t grid = (uint64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const uint64_t need = (n + kMmaThreads - 1) / kMmaThreads;
    if (grid > need) grid = need;
    kern<<<(unsigned)grid, kMmaThreads, 0, stream>>>(d.weights, d.p_in, d.latent, d.p_out, cond, z_eps, seed, offset,
                                                      n, mlv, smp);
    return cudaGetLastError();
}

// ---- shape-specialised kernels (the shapes in use: the decoder benchmark's and Table 1's) ----
// The query's row [c; z] and its eps are built in registers with compile-time indices, and rows are read and
// written with the widest aligned vector accesses; the runtime-shaped kernel above stages them through shared
// memory instead.

template <int N>
__device__ __forceinline__ void load_row(const float* __restrict__ src, float* v)
{
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int k = 0; k < N; k += 4) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(src) + k / 4);
            v[k] = a.x; v[k + 1] = a.y; v[k + 2] = a.z; v[k + 3] = a.w;
        }
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int k = 0; k < N; k += 2) {
            const float2 a = __ldg(reinterpret_cast<const float2*>(src) + k / 2);
            v[k] = a.x; v[k + 1] = a.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = __ldg(src + k);
    }
}

template <int N>
__device__ __forceinline__ void store_row(float* __restrict__ dst, const float* v)
{
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int k = 0; k < N; k += 4) reinterpret_cast<float4*>(dst)[k / 4] = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int k = 0; k < N; k += 2) reinterpret_cast<float2*>(dst)[k / 2] = make_float2(v[k], v[k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) dst[k] = v[k];
    }
}

// x[PI .. PI+L) = z and eps[0 .. P) of query q: from z_eps [n][L+P], or the query's normals from its Philox
// stream (tag 0xD0, id = offset + q; layout in decoder.cuh).
template <int PI, int L, int P, int XN>
__device__ __forceinline__ void query_normals(const float* __restrict__ z_eps, uint64_t seed, uint64_t id, uint64_t q,
                                              float (&x)[XN], float (&eps)[P])
{
    constexpr int NZ = L + P;
    float nz[(NZ + 3) / 4 * 4];
    if (z_eps) {
        load_row<NZ>(z_eps + q * NZ, nz);
    } else {
        query_normals_philox<NZ>(Stream(seed, id), 0xD0u, nz);
    }
#pragma unroll
    for (int m = 0; m < L; ++m) x[PI + m] = nz[m];
#pragma unroll
    for (int m = 0; m < P; ++m) eps[m] = nz[L + m];
}

template <int PI, int L, int P, int NTH, bool kBF16, int kSplit>
__global__ void __launch_bounds__(kMmaThreads) infer_mma_fixed(const float* __restrict__ wts,
                                                               const float* __restrict__ cond,
                                                               const float* __restrict__ z_eps, uint64_t seed,
                                                               uint64_t offset, uint64_t n, float* __restrict__ mlv,
                                                               float* __restrict__ smp)
{
    constexpr int NT3 = mmadec::n_tiles_out(P);
    __shared__ __align__(16) unsigned char wsm[mmadec::smem_bytes(P, NTH)];
    __shared__ float stage[kMmaThreads / 32][mmadec::kStageFloats];
    mmadec::stage_weights<kBF16, NTH, kSplit == 3>(wsm, wts, PI + L, P);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t n_chunks = (n + 31) / 32;
    const uint64_t warps = (uint64_t)gridDim.x * (kMmaThreads / 32);
    // the condition row of the warp's next chunk is loaded one iteration ahead (its latency hides behind the
    // current chunk's work)
    uint64_t ch = (uint64_t)blockIdx.x * (kMmaThreads / 32) + warp;
    float cnext[PI];
#pragma unroll
    for (int k = 0; k < PI; ++k) cnext[k] = 0.0f;
    if (ch * 32 + lane < n) load_row<PI>(cond + (ch * 32 + lane) * PI, cnext);
    for (; ch < n_chunks; ch += warps) {
        const uint64_t q = ch * 32 + lane;
        const bool live = q < n;
        float x[16], eps[P];
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = k < PI ? cnext[k < PI ? k : 0] : 0.0f;
#pragma unroll
        for (int k = 0; k < P; ++k) eps[k] = 0.0f;
        const uint64_t qn = q + warps * 32;
        if (qn < n) load_row<PI>(cond + qn * PI, cnext);
        if (live) query_normals<PI, L, P>(z_eps, seed, offset + q, q, x, eps);
        float y[8 * NT3];
        mmadec::warp_mlp<NT3, kSplit, kBF16, NTH>(wsm, stage[warp], x, y);
        if (live) {
            if (mlv) store_row<2 * P>(mlv + q * (2 * P), y);
            if (smp) {
                float o[P];
#pragma unroll
                for (int k = 0; k < P; ++k) o[k] = y[k] + __expf(0.5f * y[P + k]) * eps[k];
                store_row<P>(smp + q * P, o);
            }
        }
    }
}

template <typename K>
cudaError_t launch_grid(K kern, int threads, uint64_t rows_per_block, uint64_t n, cudaStream_t stream,
                        const ms_decoder& d, const float* cond, const float* z_eps, uint64_t seed, uint64_t offset,
                        float* mlv, float* smp)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    if (e != cudaSuccess) return e;
    uint64_t grid = (uint64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const uint64_t need = (n + rows_per_block - 1) / rows_per_block;
    if (grid > need) grid = need;
    kern<<<(unsigned)grid, threads, 0, stream>>>(d.weights, cond, z_eps, seed, offset, n, mlv, smp);
    return cudaGetLastError();
}

// The specialised shapes: (p_in, latent, p_out, width).
#define MS_INFER_SHAPES(X) X(4, 4, 1, 16) X(4, 4, 6, 16) X(2, 2, 1, 8) X(3, 5, 3, 16) X(7, 5, 6, 16)

// Launches the specialised kernel for d's shape and precision; returns false when the shape has none, or when
// a row pointer is not 16-byte aligned (the vector accesses need it; those calls take the runtime-shaped path).
bool launch_fixed(const ms_decoder& d, const float* cond, const float* z_eps, uint64_t seed, uint64_t offset,
                  uint64_t n, float* mlv, float* smp, cudaStream_t s, cudaError_t* err)
{
    if (((uintptr_t)cond | (uintptr_t)z_eps | (uintptr_t)mlv | (uintptr_t)smp) & 15u) return false;
#define MS_FIXED_CASE(pi, l, p, w)                                                                            \
    if (d.p_in == pi && d.latent == l && d.p_out == p && d.width == w) {                                      \
        if (d.precision == MS_FP32)                                                                            \
            *err = launch_grid(infer_mma_fixed<pi, l, p, w / 8, false, 3>, kMmaThreads, kMmaThreads, n, s, d,   \
                               cond, z_eps, seed, offset, mlv, smp);                                           \
        else if (d.precision == MS_BF16)                                                                       \
            *err = launch_grid(infer_mma_fixed<pi, l, p, w / 8, true, 2>, kMmaThreads, kMmaThreads, n, s, d,    \
                               cond, z_eps, seed, offset, mlv, smp);                                           \
        else                                                                                                   \
            *err = launch_grid(infer_mma_fixed<pi, l, p, w / 8, false, 2>, kMmaThreads, kMmaThreads, n, s, d,   \
                               cond, z_eps, seed, offset, mlv, smp);                                           \
        return true;                                                                                           \
    }
    MS_INFER_SHAPES(MS_FIXED_CASE)
#undef MS_FIXED_CASE
    return false;
}

}  // namespace dec
}  // namespace ms

extern "C" ms_status ms_cvae_infer(const ms_decoder* d, const float* cond, const float* z_eps, uint64_t seed,
                                   uint64_t offset, uint64_t n, float* out_mean_logvar, float* out_sample,
                                   void* stream)
{
    MS_NVTX("ms_cvae_infer");
    MS_CHECK_ARG(d != nullptr && d->weights != nullptr, "ms_cvae_infer: null decoder or weights");
    MS_CHECK_ARG(d->width == 8 || d->width == 16, "ms_cvae_infer: width must be 8 or 16 (got %d)", d->width);
    MS_CHECK_ARG(d->p_in >= 1 && d->latent >= 1 && d->latent <= 8 && d->p_in + d->latent <= 16,
                 "ms_cvae_infer: need 1 <= p_in, 1 <= latent <= 8, p_in + latent <= 16");
    MS_CHECK_ARG(d->p_out >= 1 && d->p_out <= 8, "ms_cvae_infer: p_out must be in 1..8");
    MS_CHECK_ARG(d->precision == MS_FP32 || d->precision == MS_FP16 || d->precision == MS_BF16,
                 "ms_cvae_infer: precision must be MS_FP32, MS_FP16 or MS_BF16");
    MS_CHECK_ARG(n == 0 || cond != nullptr, "ms_cvae_infer: cond is null");
    if (n == 0 || (out_mean_logvar == nullptr && out_sample == nullptr)) return MS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t fe = cudaSuccess;
    if (ms::dec::launch_fixed(*d, cond, z_eps, seed, offset, n, out_mean_logvar, out_sample, s, &fe)) {
        MS_CUDA(fe);
        return MS_OK;
    }
    MS_CUDA(ms::dec::launch_infer_mma(*d, cond, z_eps, seed, offset, n, out_mean_logvar, out_sample, s));
    return MS_OK;
}
