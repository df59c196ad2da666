// Warp-level CVAE decoder MLP (Sec. 3.2) on the tensor cores with mma.sync.m16n8k16 (FP32 accumulation).
//
// A warp evaluates 32 rows at once (two 16-row tiles), one row per lane:
//   y = W3 sp(W2 sp(W1 x + b1) + b2) + b3,   x in R^16 (zero padded), hidden width 8 NTH (8 or 16),
//   y in R^{8 NT3}.  A width-8 hidden layer fills the lower half of the next layer's k = 16 operand and zeros
//   the upper half.
// The weights are pre-arranged once per block in shared memory in the B-fragment order of the instruction
// (each lane loads its two 32-bit operand registers per 8-column tile with one 16-byte load), the biases
// initialise the accumulators, and the accumulator fragment of a hidden layer is, register for register, the
// A fragment of the next layer (rows g and g+8, columns 2t, 2t+1 and 2t+8, 2t+9), so Softplus is applied in
// place and no data moves between layers.  Inputs and outputs pass through a per-warp shared staging tile.
//
// Precision: kSplit = 3 splits activations and weights into a half-precision head and tail and sums
// head*head + head*tail + tail*head, which keeps about 22 significant bits (single-precision-like results);
// kSplit = 2 splits the activations only (inputs and hidden layers carried as head + tail, weights rounded
// once to half precision), so the error is that of the rounded weights; kSplit = 1 is plain half precision.
// Half is FP16 (kBF16 = false) or BF16.  Accumulation is FP32 throughout.
//
// Softplus in base 2: every decoder evaluates its hidden layers on pre-activations scaled by log2(e),
// a' = a log2(e), where sp(a) = ln(2) sp2(a') with sp2(a') = max(a', 0) + log2(1 + 2^-|a'|): each hidden unit
// then costs 2^x, log2 and three additions, without the two scalings that sp(a) = max(a, 0) + ln(1 + e^-|a|)
// needs on the special-function unit.  The scalings are folded in where they cost nothing: the first two
// layers' biases are staged times log2(e); the first hidden layer's ln(2) cancels the second layer's log2(e),
// so the second layer's weights stay as they are.  The first layer's log2(e) and the last hidden layer's ln(2)
// are folded into the first and third layers' weights with kSplit = 3 (weights split into head and tail, so
// the scaled weights are exact to about 22 bits); with the half-precision weights of kSplit <= 2 the scaled
// weights would round differently from the weights themselves, so there the input row is multiplied by
// log2(e) before it is split and the last hidden layer's outputs by ln(2) (FP32 values, carried as head and
// tail).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ms_device.cuh"

namespace ms {
namespace mmadec {

constexpr int kStageStride = 17;                         // floats per staged row (odd: no bank conflicts)
constexpr int kStageFloats = 32 * kStageStride;          // one warp's staging tile

__host__ __device__ constexpr int n_tiles_out(int p_out) { return (2 * p_out + 7) / 8; }
// shared layout of one decoder with NTH hidden tiles (width 8 NTH): fragments [NTH + NTH + NT3][32] uint4, then
// biases [8 NTH + 8 NTH + 8 NT3] floats
__host__ __device__ constexpr int frag_tiles(int p_out, int nth = 2) { return 2 * nth + n_tiles_out(p_out); }
__host__ __device__ constexpr int smem_bytes(int p_out, int nth = 2)
{
    return frag_tiles(p_out, nth) * 32 * 16 + (16 * nth + 8 * n_tiles_out(p_out)) * 4;
}

template <bool kBF16>
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    if constexpr (kBF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
}

template <bool kBF16>
__device__ __forceinline__ float2 unpack2(uint32_t v)
{
    if constexpr (kBF16) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v));
    } else {
        return __half22float2(*reinterpret_cast<const __half2*>(&v));
    }
}

// head = round(a, b); tail = round((a, b) - head)
template <bool kBF16>
__device__ __forceinline__ void split2(float a, float b, uint32_t& head, uint32_t& tail)
{
    head = pack2<kBF16>(a, b);
    const float2 h = unpack2<kBF16>(head);
    tail = pack2<kBF16>(a - h.x, b - h.y);
}

template <bool kBF16>
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    if constexpr (kBF16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// Block-wide: packed float weights W1[w][k_in] b1 W2[w][w] b2 W3[2p][w] b3 (w = 8 NTH) -> fragment layout at
// `dst`.  For 8-column tile j and lane (g = lane / 4, t = lane % 4) the B operand holds rows k = 2t, 2t+1 (b0)
// and 2t+8, 2t+9 (b1) of column n = 8j + g, i.e. W[n][k] (zero for k >= K); stored as
// {b0 head, b1 head, b0 tail, b1 tail}.  The scalings of the base-2 Softplus (see above): biases of the first
// two layers times log2(e) always; with kScaleW (kSplit = 3) also the first layer's weights times log2(e) and
// the third layer's times ln(2).
constexpr float kLog2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;

template <bool kBF16, int NTH = 2, bool kScaleW = false>
__device__ void stage_weights(unsigned char* dst, const float* __restrict__ g, int k_in, int p_out)
{
    const float wscale[3] = {kScaleW ? kLog2e : 1.0f, 1.0f, kScaleW ? kLn2 : 1.0f};
    const float bscale[3] = {kLog2e, kLog2e, 1.0f};
    constexpr int w = 8 * NTH;
    const int nt3 = n_tiles_out(p_out);
    uint4* frag = reinterpret_cast<uint4*>(dst);
    float* bias = reinterpret_cast<float*>(dst + frag_tiles(p_out, NTH) * 32 * 16);
    const float* W[3] = {g, g + w * k_in + w, g + w * k_in + w + w * w + w};
    const float* Bv[3] = {g + w * k_in, g + w * k_in + w + w * w, g + w * k_in + w + w * w + w + 2 * p_out * w};
    const int K[3] = {k_in, w, w};
    const int N[3] = {w, w, 2 * p_out};
    const int T0[3] = {0, NTH, 2 * NTH};
    const int total = frag_tiles(p_out, NTH) * 32;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int tile = e >> 5, lane = e & 31;
        const int layer = tile < NTH ? 0 : (tile < 2 * NTH ? 1 : 2);
        const int j = tile - T0[layer];
        const int n = 8 * j + (lane >> 2), t = lane & 3;
        auto w = [&](int k) -> float {
            return (n < N[layer] && k < K[layer]) ? wscale[layer] * W[layer][n * K[layer] + k] : 0.0f;
        };
        float v[4] = {w(2 * t), w(2 * t + 1), w(2 * t + 8), w(2 * t + 9)};
        uint32_t h0, l0, h1, l1;
        {
            h0 = pack2<kBF16>(v[0], v[1]);
            const float2 a = unpack2<kBF16>(h0);
            l0 = pack2<kBF16>(v[0] - a.x, v[1] - a.y);
            h1 = pack2<kBF16>(v[2], v[3]);
            const float2 b = unpack2<kBF16>(h1);
            l1 = pack2<kBF16>(v[2] - b.x, v[3] - b.y);
        }
        frag[e] = make_uint4(h0, h1, l0, l1);
    }
    for (int e = threadIdx.x; e < 2 * w + 8 * nt3; e += blockDim.x) {
        if (e < w) bias[e] = bscale[0] * Bv[0][e];
        else if (e < 2 * w) bias[e] = bscale[1] * Bv[1][e - w];
        else bias[e] = (e - 2 * w) < 2 * p_out ? Bv[2][e - 2 * w] : 0.0f;
    }
}

// One layer for MT 16-row tiles: acc = bias + A W^T, A given as half-precision head (and tail) fragments.
template <int NT, int kSplit, bool kBF16, int MT = 2>
__device__ __forceinline__ void layer(const uint32_t (&ah)[MT][4], const uint32_t (&al)[MT][4],
                                      const uint4* __restrict__ frag, const float* __restrict__ bias, int lane,
                                      float (&acc)[MT][NT][4])
{
    const int t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const uint4 w = frag[nt * 32 + lane];
        const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            acc[mt][nt][0] = b0; acc[mt][nt][1] = b1; acc[mt][nt][2] = b0; acc[mt][nt][3] = b1;
            if (kSplit >= 2) mma<kBF16>(acc[mt][nt], al[mt], w.x, w.y);
            if (kSplit == 3) mma<kBF16>(acc[mt][nt], ah[mt], w.z, w.w);
            mma<kBF16>(acc[mt][nt], ah[mt], w.x, w.y);
        }
    }
}

// sp2(a) = max(a, 0) + log2(1 + 2^-|a|): Softplus in base 2 on the special-function unit's 2^x and log2.
__device__ __forceinline__ float softplus2(float a)
{
    float e, l;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-fabsf(a)));
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(1.0f + e));
    return fmaxf(a, 0.0f) + l;
}

// Softplus (base 2, on the scaled pre-activations) of an 8 NTH-wide hidden layer, re-packed as the next
// layer's A fragments (head and tail); with NTH = 1 the upper k half (columns 8..15) is zero.  kOutScale: the
// last hidden layer with half-precision weights, whose outputs are multiplied by ln(2) (see above).
template <int kSplit, bool kBF16, int NTH = 2, int MT = 2, bool kOutScale = false>
__device__ __forceinline__ void hidden_to_a(const float (&acc)[MT][NTH][4], uint32_t (&ah)[MT][4],
                                            uint32_t (&al)[MT][4])
{
    auto sp = [](float a) -> float { return kOutScale ? kLn2 * softplus2(a) : softplus2(a); };
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
        float s[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            s[i] = sp(acc[mt][0][i]);
            s[4 + i] = NTH == 2 ? sp(acc[mt][NTH - 1][i]) : 0.0f;
        }
        if (kSplit >= 2) {
            split2<kBF16>(s[0], s[1], ah[mt][0], al[mt][0]);
            split2<kBF16>(s[2], s[3], ah[mt][1], al[mt][1]);
            split2<kBF16>(s[4], s[5], ah[mt][2], al[mt][2]);
            split2<kBF16>(s[6], s[7], ah[mt][3], al[mt][3]);
        } else {
            ah[mt][0] = pack2<kBF16>(s[0], s[1]);
            ah[mt][1] = pack2<kBF16>(s[2], s[3]);
            ah[mt][2] = pack2<kBF16>(s[4], s[5]);
            ah[mt][3] = pack2<kBF16>(s[6], s[7]);
        }
    }
}

// The whole MLP for the warp's 32 rows; every lane of the warp must call it (it synchronises the warp).
// x: this lane's input row (16 values, zero padded); y: this lane's 8*NT3 outputs (mu then log Sigma).
template <int NT3, int kSplit, bool kBF16, int NTH = 2>
__device__ __forceinline__ void warp_mlp(const unsigned char* __restrict__ wsm, float* __restrict__ stage,
                                         const float (&x)[16], float (&y)[8 * NT3])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint4* frag = reinterpret_cast<const uint4*>(wsm);
    const float* bias = reinterpret_cast<const float*>(wsm + (2 * NTH + NT3) * 32 * 16);
    constexpr float kIn = kSplit == 3 ? 1.0f : kLog2e;     // the first layer's log2(e), on the input row
#pragma unroll
    for (int j = 0; j < 16; ++j) stage[lane * kStageStride + j] = kIn * x[j];
    __syncwarp();
    uint32_t ah[2][4], al[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const float* r0 = stage + (16 * mt + g) * kStageStride;
        const float* r1 = r0 + 8 * kStageStride;
        split2<kBF16>(r0[2 * t], r0[2 * t + 1], ah[mt][0], al[mt][0]);
        split2<kBF16>(r1[2 * t], r1[2 * t + 1], ah[mt][1], al[mt][1]);
        split2<kBF16>(r0[2 * t + 8], r0[2 * t + 9], ah[mt][2], al[mt][2]);
        split2<kBF16>(r1[2 * t + 8], r1[2 * t + 9], ah[mt][3], al[mt][3]);
    }
    __syncwarp();
    float h[2][NTH][4];
    layer<NTH, kSplit, kBF16>(ah, al, frag, bias, lane, h);
    hidden_to_a<kSplit, kBF16, NTH>(h, ah, al);
    layer<NTH, kSplit, kBF16>(ah, al, frag + NTH * 32, bias + 8 * NTH, lane, h);
    hidden_to_a<kSplit, kBF16, NTH, 2, kSplit != 3>(h, ah, al);
    float o[2][NT3][4];
    layer<NT3, kSplit, kBF16>(ah, al, frag + 2 * NTH * 32, bias + 16 * NTH, lane, o);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT3; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 16 * mt + g + (i >= 2 ? 8 : 0);
                const int c = 8 * nt + 2 * t + (i & 1);
                stage[r * kStageStride + c] = o[mt][nt][i];
            }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 8 * NT3; ++j) y[j] = stage[lane * kStageStride + j];
    __syncwarp();
}

// The MLP for the 16 rows of one tile, staged by row index instead of by lane: a lane with `active` set
// supplies input row `row` (0..15) and receives that row's outputs; other lanes supply nothing and get zeros.
// Rows no active lane supplied carry whatever the staging tile held: every output row depends on its own input
// row only, so those rows are computed and ignored.  Every lane of the warp must call it.  Used where fewer
// than half a warp's lanes have a query: the work is that of one tile instead of two.
// KIN: the number of input columns in use (x[j] = 0 for j >= KIN is assumed); with KIN <= 8 the upper half of
// the input tile is known to be zero and is neither staged nor loaded.  KOUT: the outputs the caller uses (the
// rest of y is zero).
template <int NT3, int kSplit, bool kBF16, int NTH = 2, int KIN = 16, int KOUT = 8 * NT3>
__device__ __forceinline__ void warp_mlp_rows16(const unsigned char* __restrict__ wsm, float* __restrict__ stage,
                                                const float (&x)[16], float (&y)[8 * NT3], int row, bool active)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint4* frag = reinterpret_cast<const uint4*>(wsm);
    const float* bias = reinterpret_cast<const float*>(wsm + (2 * NTH + NT3) * 32 * 16);
    constexpr int kCols = KIN <= 8 ? 8 : 16;
    constexpr float kIn = kSplit == 3 ? 1.0f : kLog2e;     // the first layer's log2(e), on the input row
    if (active) {
#pragma unroll
        for (int j = 0; j < kCols; ++j) stage[row * kStageStride + j] = kIn * x[j];
    }
    __syncwarp();
    uint32_t ah[1][4], al[1][4];
    {
        const float* r0 = stage + g * kStageStride;
        const float* r1 = r0 + 8 * kStageStride;
        split2<kBF16>(r0[2 * t], r0[2 * t + 1], ah[0][0], al[0][0]);
        split2<kBF16>(r1[2 * t], r1[2 * t + 1], ah[0][1], al[0][1]);
        if constexpr (kCols == 16) {
            split2<kBF16>(r0[2 * t + 8], r0[2 * t + 9], ah[0][2], al[0][2]);
            split2<kBF16>(r1[2 * t + 8], r1[2 * t + 9], ah[0][3], al[0][3]);
        } else {
            ah[0][2] = al[0][2] = ah[0][3] = al[0][3] = 0u;
        }
    }
    __syncwarp();
    float h[1][NTH][4];
    layer<NTH, kSplit, kBF16, 1>(ah, al, frag, bias, lane, h);
    hidden_to_a<kSplit, kBF16, NTH, 1>(h, ah, al);
    layer<NTH, kSplit, kBF16, 1>(ah, al, frag + NTH * 32, bias + 8 * NTH, lane, h);
    hidden_to_a<kSplit, kBF16, NTH, 1, kSplit != 3>(h, ah, al);
    float o[1][NT3][4];
    layer<NT3, kSplit, kBF16, 1>(ah, al, frag + 2 * NTH * 32, bias + 16 * NTH, lane, o);
#pragma unroll
    for (int nt = 0; nt < NT3; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = g + (i >= 2 ? 8 : 0);
            const int c = 8 * nt + 2 * t + (i & 1);
            stage[r * kStageStride + c] = o[0][nt][i];
        }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 8 * NT3; ++j) y[j] = (active && j < KOUT) ? stage[row * kStageStride + j] : 0.0f;
    __syncwarp();
}

}  // namespace mmadec
}  // namespace ms
