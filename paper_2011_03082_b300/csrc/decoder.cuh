// CVAE decoder MLP (Sec. 3.2, Fig. 3b): three weight layers, Softplus between hidden layers, linear output
// (mu, log Sigma).  Single-precision, one query per thread, weights in shared memory.
//
// Shared-memory layout (floats) for hidden width W, transposed so that one input's weights to all outputs are
// contiguous and every weight load is a 16-byte broadcast (all lanes read the same address):
//   W1t[IN4][W] b1[W] W2t[W][W] b2[W] W3t[W][O4] b3[O4]      (O4 = 2P rounded up to 4, zero padded)
// The layer loops run input-outer / output-inner, so only the W accumulators and one weight row are live.
#pragma once

#include "ms_device.cuh"

namespace ms {
namespace dec {

__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }

template <int W>
__host__ __device__ constexpr int smem_floats(int in4, int p)
{
    return in4 * W + W + W * W + W + W * pad4(2 * p) + pad4(2 * p);
}

// Copies packed weights (W1[W][in] b1 W2[W][W] b2 W3[2p][W] b3) into the transposed shared layout.
template <int W>
__device__ __forceinline__ void stage_weights(float* s, const float* __restrict__ g, int in, int in4, int p)
{
    const int o4 = pad4(2 * p);
    float* W1t = s;
    float* b1 = W1t + in4 * W;
    float* W2t = b1 + W;
    float* b2 = W2t + W * W;
    float* W3t = b2 + W;
    float* b3 = W3t + W * o4;
    const float* gW1 = g;
    const float* gb1 = gW1 + W * in;
    const float* gW2 = gb1 + W;
    const float* gb2 = gW2 + W * W;
    const float* gW3 = gb2 + W;
    const float* gb3 = gW3 + 2 * p * W;
    for (int t = threadIdx.x; t < in4 * W; t += blockDim.x) {
        const int k = t / W, o = t - k * W;
        W1t[t] = k < in ? gW1[o * in + k] : 0.0f;
    }
    for (int t = threadIdx.x; t < W * W; t += blockDim.x) {
        const int k = t / W, o = t - k * W;
        W2t[t] = gW2[o * W + k];
    }
    for (int t = threadIdx.x; t < W * o4; t += blockDim.x) {
        const int k = t / o4, o = t - k * o4;
        W3t[t] = o < 2 * p ? gW3[o * W + k] : 0.0f;
    }
    for (int t = threadIdx.x; t < W; t += blockDim.x) {
        b1[t] = gb1[t];
        b2[t] = gb2[t];
    }
    for (int t = threadIdx.x; t < o4; t += blockDim.x) b3[t] = t < 2 * p ? gb3[t] : 0.0f;
}

template <int K, int O>
__device__ __forceinline__ void dense(const float* __restrict__ Wt, const float* __restrict__ b, const float (&x)[K],
                                      float (&acc)[O])
{
#pragma unroll
    for (int o = 0; o < O; o += 4) {
        const float4 v = *reinterpret_cast<const float4*>(b + o);
        acc[o] = v.x; acc[o + 1] = v.y; acc[o + 2] = v.z; acc[o + 3] = v.w;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 0; o < O; o += 4) {
            const float4 w = *reinterpret_cast<const float4*>(Wt + k * O + o);
            acc[o] = fmaf(w.x, x[k], acc[o]);
            acc[o + 1] = fmaf(w.y, x[k], acc[o + 1]);
            acc[o + 2] = fmaf(w.z, x[k], acc[o + 2]);
            acc[o + 3] = fmaf(w.w, x[k], acc[o + 3]);
        }
    }
}

// y = W3 sp(W2 sp(W1 x + b1) + b2) + b3; x has IN4 entries (zero padded), y has pad4(2P) entries.
template <int IN4, int P, int W>
__device__ __forceinline__ void mlp(const float* __restrict__ s, const float (&x)[IN4], float (&y)[pad4(2 * P)])
{
    constexpr int O4 = pad4(2 * P);
    const float* W1t = s;
    const float* b1 = W1t + IN4 * W;
    const float* W2t = b1 + W;
    const float* b2 = W2t + W * W;
    const float* W3t = b2 + W;
    const float* b3 = W3t + W * O4;
    float h[W], g[W];
    dense<IN4, W>(W1t, b1, x, h);
#pragma unroll
    for (int o = 0; o < W; ++o) h[o] = softplus(h[o]);
    dense<W, W>(W2t, b2, h, g);
#pragma unroll
    for (int o = 0; o < W; ++o) g[o] = softplus(g[o]);
    dense<W, O4>(W3t, b3, g, y);
}

// Standard normals 4j..4j+3 of a query: counter (j, id_lo, id_hi, tag), Box-Muller on word pairs.
__device__ __forceinline__ float4 normals4(const Stream& st, uint32_t j, uint32_t tag)
{
    const Words w = st.at(j, tag);
    const float2 a = box_muller(w.w0, w.w1), b = box_muller(w.w2, w.w3);
    return make_float4(a.x, a.y, b.x, b.y);
}

}  // namespace dec
}  // namespace ms
