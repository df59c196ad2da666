// CVAE training (Sec. 3.2): negative ELBO, its analytic gradient and Adam, hand-written.
//
//   encoder  [x ; c] -> 16 -> 16 -> (mu_e, log Sigma_e) in R^L       (Softplus between hidden layers)
//   z = mu_e + exp(lv_e / 2) eps
//   decoder  [c ; z] -> 16 -> 16 -> (mu_d, log Sigma_d) in R^P
//   loss = mean_b [ 0.5 sum_d (lv_d + (x_d - mu_d)^2 e^{-lv_d} + ln 2 pi) + 0.5 sum_l (mu_l^2 + e^{lv_l} - lv_l - 1) ]
//
// Kernel design:
//  * fwd_bwd: one sample per thread, 128 samples per block.  Forward and backward run in registers; the
//    layer inputs and the back-propagated deltas of every layer are staged in shared memory (rows padded to
//    an odd stride), after which the block forms its partial weight gradient sum_s delta[s][o] * in[s][k]:
//    in FP32 on the tensor cores (each warp takes whole layers, 3xTF32 m16n8k8 products with the samples as
//    the k dimension), in BF16 mode with FFMA register tiles; either way in a fixed order.  Per-block
//    partials go to the workspace: no floating-point atomics anywhere, so the gradient is bit-reproducible.
//  * reduce: each block sums 32 parameters' block partials, eight warps over interleaved block rows, the
//    warp sums added in warp order, and writes the gradient and the loss terms.
//  * adam: element-wise bias-corrected Adam (AdamW decay when weight_decay > 0).
// Precision: MS_FP32, or MS_BF16 — weight matrices and every layer's input rounded to BF16 (round to nearest
// even) in the forward and backward passes, with biases, pre-activations, accumulation, losses, gradients,
// master weights and Adam in FP32 (mixed-precision training numerics).
#include <cmath>

#include <cuda_bf16.h>
#include <type_traits>

#include "ms_device.cuh"

namespace ms {
namespace train {

constexpr int kSamples = 128;

// Hidden width kW and latent size kL are shape parameters (Table 1 uses W 8 or 16, L 2 or 5).
template <int PI, int PO, int kW, int kL>
struct Shape {
    static constexpr int W = kW, L = kL;
    static constexpr int IE = PO + PI;                // encoder input
    static constexpr int ID = PI + kL;                // decoder input
    // packed parameter offsets: encoder E1 e1 E2 e2 E3 e3, then decoder D1 d1 D2 d2 D3 d3
    static constexpr int E1 = 0, e1 = E1 + kW * IE, E2 = e1 + kW, e2 = E2 + kW * kW, E3 = e2 + kW,
                         e3 = E3 + 2 * kL * kW, D1 = e3 + 2 * kL, d1 = D1 + kW * ID, D2 = d1 + kW,
                         d2 = D2 + kW * kW, D3 = d2 + kW, d3 = D3 + 2 * PO * kW, NP = d3 + 2 * PO;
    // shared staging: per sample, the inputs and deltas of the six layers; rows of stride 17 (odd), and slots
    // SLOT floats apart (not a multiple of 32, so equal columns of different slots fall in different banks)
    static constexpr int R = 17;
    static constexpr int SLOT = kSamples * R + 5;
    enum Slot { IN1E, H1E, H2E, IN1D, H1D, H2D, DA1E, DA2E, DOE, DA1D, DA2D, DY, NSLOT };
    // the six weight matrices in shared memory after the slots, rows padded to a multiple of 4 (float4 loads)
    static constexpr int P4(int k) { return (k + 3) & ~3; }
    static constexpr int sE1 = 0, sE2 = sE1 + kW * P4(IE), sE3 = sE2 + kW * P4(kW), sD1 = sE3 + 2 * kL * P4(kW),
                         sD2 = sD1 + kW * P4(ID), sD3 = sD2 + kW * P4(kW), SW = sD3 + 2 * PO * P4(kW);
};

__device__ __forceinline__ float sigmoidf_fast(float a) { return __fdividef(1.0f, 1.0f + __expf(-a)); }

// 3xTF32: x = head + tail with both rounded to TF32 (10-bit mantissa, FP32 exponent range); head*head +
// head*tail + tail*head keeps about 21 significant bits of every product, with FP32 accumulation.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo)
{
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(x - __uint_as_float(hi)));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// value as the layer sees it: unchanged in FP32, rounded to BF16 (nearest even) in the BF16 variant
template <bool kBF16>
__device__ __forceinline__ float rq(float x)
{
    if constexpr (kBF16) return __bfloat162float(__float2bfloat16_rn(x));
    else return x;
}

// Weights Ws: shared memory, row-major [O][K4] with K4 = K rounded up to 4 (zero padded); every lane of a warp
// reads the same row, so each float4 load is a broadcast serving four FMAs.  Sums run over k in order.
template <int K, int O, bool kBF16>
__device__ __forceinline__ void fwd_layer(const float* __restrict__ Ws, const float* __restrict__ b,
                                          const float (&x)[K], float (&a)[O])
{
    constexpr int K4 = (K + 3) & ~3;
#pragma unroll
    for (int o = 0; o < O; ++o) {
        float acc = __ldg(b + o);
#pragma unroll
        for (int k = 0; k < K4; k += 4) {
            const float4 w = *reinterpret_cast<const float4*>(Ws + o * K4 + k);
            const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (k + j < K) acc = fmaf(rq<kBF16>(wv[j]), x[k + j], acc);
        }
        a[o] = acc;
    }
}

// dx = W^T da
template <int K, int O, bool kBF16>
__device__ __forceinline__ void bwd_layer(const float* __restrict__ Ws, const float (&da)[O], float (&dx)[K])
{
    constexpr int K4 = (K + 3) & ~3;
#pragma unroll
    for (int k = 0; k < K; ++k) dx[k] = 0.0f;
#pragma unroll
    for (int o = 0; o < O; ++o)
#pragma unroll
        for (int k = 0; k < K4; k += 4) {
            const float4 w = *reinterpret_cast<const float4*>(Ws + o * K4 + k);
            const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (k + j < K) dx[k + j] = fmaf(rq<kBF16>(wv[j]), da[o], dx[k + j]);
        }
}

// Copies one [O][K] weight matrix into the padded shared layout.
template <int O, int K>
__device__ __forceinline__ void stage_matrix(float* __restrict__ dst, const float* __restrict__ src)
{
    constexpr int K4 = (K + 3) & ~3;
    for (int i = threadIdx.x; i < O * K4; i += blockDim.x) {
        const int o = i / K4, k = i - o * K4;
        dst[i] = k < K ? src[o * K + k] : 0.0f;
    }
}

// kGrad = false: the loss alone (ms_cvae_forward): no backward pass and no staging slots in shared memory; only
// the two loss partials of the block are written.
template <int PI, int PO, int kW, int kL, bool kBF16, bool kGrad = true>
__global__ void __launch_bounds__(kSamples) fwd_bwd(const float* __restrict__ prm, const float* __restrict__ X,
                                                    const float* __restrict__ Cc, const float* __restrict__ EPS,
                                                    uint64_t B, uint64_t seed, uint64_t step,
                                                    float* __restrict__ partial)
{
    using S = Shape<PI, PO, kW, kL>;
    extern __shared__ float sm[];
    const int t = threadIdx.x;
    const uint64_t b = (uint64_t)blockIdx.x * kSamples + t;
    const bool live = b < B;
    float* row_base = sm;   // [NSLOT][SLOT]: sample s of a slot at s * R
    auto row = [&](int slot, int s) -> float* { return row_base + (size_t)slot * S::SLOT + (size_t)s * S::R; };
    __shared__ float s_rec[kSamples / 32], s_kl[kSamples / 32];
    float* ws = sm + (kGrad ? S::NSLOT * S::SLOT : 0);    // padded weight matrices
    stage_matrix<kW, S::IE>(ws + S::sE1, prm + S::E1);
    stage_matrix<kW, kW>(ws + S::sE2, prm + S::E2);
    stage_matrix<2 * kL, kW>(ws + S::sE3, prm + S::E3);
    stage_matrix<kW, S::ID>(ws + S::sD1, prm + S::D1);
    stage_matrix<kW, kW>(ws + S::sD2, prm + S::D2);
    stage_matrix<2 * PO, kW>(ws + S::sD3, prm + S::D3);
    __syncthreads();

    // ---------------- forward ----------------
    float xin[S::IE], c[PI], x[PO];
#pragma unroll
    for (int j = 0; j < PO; ++j) x[j] = live ? X[b * PO + j] : 0.0f;
#pragma unroll
    for (int j = 0; j < PI; ++j) c[j] = live ? Cc[b * PI + j] : 0.0f;
#pragma unroll
    for (int j = 0; j < PO; ++j) xin[j] = rq<kBF16>(x[j]);
#pragma unroll
    for (int j = 0; j < PI; ++j) xin[PO + j] = rq<kBF16>(c[j]);
    float eps[kL];
    if (EPS) {
#pragma unroll
        for (int l = 0; l < kL; ++l) eps[l] = live ? EPS[b * kL + l] : 0.0f;
    } else {
        // normals 4j..4j+3 from counter (j, b, step, 0xE0)
        const Stream st(seed, (step << 32) | (b & 0xffffffffull));
#pragma unroll
        for (int j = 0; 4 * j < kL; ++j) {
            const Words w = st.at((uint32_t)j, 0xE0u);
            const float2 p0 = box_muller(w.w0, w.w1), p1 = box_muller(w.w2, w.w3);
            const float v[4] = {p0.x, p0.y, p1.x, p1.y};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (4 * j + i < kL) eps[4 * j + i] = v[i];
        }
    }
    float a1e[kW], h1e[kW], a2e[kW], h2e[kW], oe[2 * kL];
    fwd_layer<S::IE, kW, kBF16>(ws + S::sE1, prm + S::e1, xin, a1e);
#pragma unroll
    for (int o = 0; o < kW; ++o) h1e[o] = rq<kBF16>(softplus(a1e[o]));
    fwd_layer<kW, kW, kBF16>(ws + S::sE2, prm + S::e2, h1e, a2e);
#pragma unroll
    for (int o = 0; o < kW; ++o) h2e[o] = rq<kBF16>(softplus(a2e[o]));
    fwd_layer<kW, 2 * kL, kBF16>(ws + S::sE3, prm + S::e3, h2e, oe);
    float sd_e[kL], z[kL];
#pragma unroll
    for (int l = 0; l < kL; ++l) {
        sd_e[l] = __expf(0.5f * oe[kL + l]);
        z[l] = oe[l] + sd_e[l] * eps[l];
    }
    float din[S::ID];
#pragma unroll
    for (int j = 0; j < PI; ++j) din[j] = rq<kBF16>(c[j]);
#pragma unroll
    for (int l = 0; l < kL; ++l) din[PI + l] = rq<kBF16>(z[l]);
    float a1d[kW], h1d[kW], a2d[kW], h2d[kW], y[2 * PO];
    fwd_layer<S::ID, kW, kBF16>(ws + S::sD1, prm + S::d1, din, a1d);
#pragma unroll
    for (int o = 0; o < kW; ++o) h1d[o] = rq<kBF16>(softplus(a1d[o]));
    fwd_layer<kW, kW, kBF16>(ws + S::sD2, prm + S::d2, h1d, a2d);
#pragma unroll
    for (int o = 0; o < kW; ++o) h2d[o] = rq<kBF16>(softplus(a2d[o]));
    fwd_layer<kW, 2 * PO, kBF16>(ws + S::sD3, prm + S::d3, h2d, y);

    const float invB = 1.0f / (float)B;
    float rec = 0.0f, kl = 0.0f;
    float dy[2 * PO];
#pragma unroll
    for (int d = 0; d < PO; ++d) {
        const float r = x[d] - y[d];
        const float iv = __expf(-y[PO + d]);
        rec += 0.5f * (y[PO + d] + r * r * iv + 1.8378770664093453f);
        dy[d] = live ? -r * iv * invB : 0.0f;
        dy[PO + d] = live ? 0.5f * (1.0f - r * r * iv) * invB : 0.0f;
    }
#pragma unroll
    for (int l = 0; l < kL; ++l) kl += 0.5f * (oe[l] * oe[l] + sd_e[l] * sd_e[l] - oe[kL + l] - 1.0f);

    const float m = live ? 1.0f : 0.0f;
    if constexpr (kGrad) {
        // ---------------- backward ----------------
        float dh[kW], da2d[kW], da1d[kW], ddin[S::ID];
        bwd_layer<kW, 2 * PO, kBF16>(ws + S::sD3, dy, dh);
#pragma unroll
        for (int o = 0; o < kW; ++o) da2d[o] = dh[o] * sigmoidf_fast(a2d[o]);
        bwd_layer<kW, kW, kBF16>(ws + S::sD2, da2d, dh);
#pragma unroll
        for (int o = 0; o < kW; ++o) da1d[o] = dh[o] * sigmoidf_fast(a1d[o]);
        bwd_layer<S::ID, kW, kBF16>(ws + S::sD1, da1d, ddin);
        float doe[2 * kL];
#pragma unroll
        for (int l = 0; l < kL; ++l) {
            const float dz = ddin[PI + l];
            doe[l] = live ? dz + oe[l] * invB : 0.0f;
            doe[kL + l] = live ? dz * eps[l] * 0.5f * sd_e[l] + 0.5f * (sd_e[l] * sd_e[l] - 1.0f) * invB : 0.0f;
        }
        float da2e[kW], da1e[kW];
        bwd_layer<kW, 2 * kL, kBF16>(ws + S::sE3, doe, dh);
#pragma unroll
        for (int o = 0; o < kW; ++o) da2e[o] = dh[o] * sigmoidf_fast(a2e[o]);
        bwd_layer<kW, kW, kBF16>(ws + S::sE2, da2e, dh);
#pragma unroll
        for (int o = 0; o < kW; ++o) da1e[o] = dh[o] * sigmoidf_fast(a1e[o]);

        // ---------------- stage layer inputs and deltas ----------------
#pragma unroll
        for (int k = 0; k < S::IE; ++k) row(S::IN1E, t)[k] = xin[k] * m;
#pragma unroll
        for (int k = 0; k < kW; ++k) {
            row(S::H1E, t)[k] = h1e[k] * m;
            row(S::H2E, t)[k] = h2e[k] * m;
            row(S::H1D, t)[k] = h1d[k] * m;
            row(S::H2D, t)[k] = h2d[k] * m;
            row(S::DA1E, t)[k] = da1e[k];
            row(S::DA2E, t)[k] = da2e[k];
            row(S::DA1D, t)[k] = da1d[k];
            row(S::DA2D, t)[k] = da2d[k];
        }
#pragma unroll
        for (int k = 0; k < S::ID; ++k) row(S::IN1D, t)[k] = din[k] * m;
#pragma unroll
        for (int k = 0; k < 2 * kL; ++k) row(S::DOE, t)[k] = doe[k];
#pragma unroll
        for (int k = 0; k < 2 * PO; ++k) row(S::DY, t)[k] = dy[k];
    }
    // loss partials (fixed-order warp and block sums)
    rec *= m;
    kl *= m;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        rec += __shfl_xor_sync(0xffffffffu, rec, off);
        kl += __shfl_xor_sync(0xffffffffu, kl, off);
    }
    if ((t & 31) == 0) { s_rec[t >> 5] = rec; s_kl[t >> 5] = kl; }
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * (S::NP + 2);
    if constexpr (kGrad) {
        // ---------------- block gradient: 4 x 4 register tiles, samples in order ----------------
        // Work items: per layer, the ceil(O/4) x ceil(K/4) tiles of dW = sum_s delta_s x_s^T and the ceil(O/4) 4-wide
        // tiles of db = sum_s delta_s.  Each parameter is summed over the block's samples in sample order (one FMA or
        // add per sample), exactly as a one-thread-per-parameter loop would.  Tile entries past O or K read row
        // padding and are not stored.
        auto tiles = [&](auto O_, auto K_, int dslot, int islot, int bW, int bb, int item) {
            constexpr int O = decltype(O_)::value, K = decltype(K_)::value;
            constexpr int TO = (O + 3) / 4, TK = (K + 3) / 4;
            const float* dr = row(dslot, 0);
            if (item < TO * TK) {
                const int o0 = 4 * (item / TK), k0 = 4 * (item % TK);
                const float* xr = row(islot, 0) + k0;
                dr += o0;
                float acc[4][4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
                for (int smp = 0; smp < kSamples; ++smp) {
                    const float* d = dr + smp * S::R;
                    const float* x = xr + smp * S::R;
                    const float d4[4] = {d[0], d[1], d[2], d[3]}, x4[4] = {x[0], x[1], x[2], x[3]};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(d4[i], x4[j], acc[i][j]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (o0 + i < O && k0 + j < K) out[bW + (o0 + i) * K + k0 + j] = acc[i][j];
            } else {
                const int o0 = 4 * (item - TO * TK);
                dr += o0;
                float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 4
                for (int smp = 0; smp < kSamples; ++smp) {
                    const float* d = dr + smp * S::R;
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[i] += d[i];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (o0 + i < O) out[bb + o0 + i] = acc[i];
            }
        };
        using IE = std::integral_constant<int, S::IE>;
        using ID = std::integral_constant<int, S::ID>;
        using W_ = std::integral_constant<int, kW>;
        using L2 = std::integral_constant<int, 2 * kL>;
        using P2 = std::integral_constant<int, 2 * PO>;
        constexpr int T1 = ((kW + 3) / 4) * ((S::IE + 3) / 4) + (kW + 3) / 4;
        constexpr int T2 = ((kW + 3) / 4) * ((kW + 3) / 4) + (kW + 3) / 4;
        constexpr int T3 = ((2 * kL + 3) / 4) * ((kW + 3) / 4) + (2 * kL + 3) / 4;
        constexpr int T4 = ((kW + 3) / 4) * ((S::ID + 3) / 4) + (kW + 3) / 4;
        constexpr int T6 = ((2 * PO + 3) / 4) * ((kW + 3) / 4) + (2 * PO + 3) / 4;
        constexpr int B1 = T1, B2 = B1 + T2, B3 = B2 + T3, B4 = B3 + T4, B5 = B4 + T2, B6 = B5 + T6;
        // FP32: each warp forms whole layers' dW = D^T X and db = D^T 1 on the tensor cores (3xTF32, m16n8k8,
        // the block's 128 samples as the k dimension in order); the output rows o >= O and columns k >= K read row
        // padding and are not stored.  BF16 keeps the FFMA tiles above.
        auto mma_grad = [&](auto O_, auto K_, int dslot, int islot, int bW, int bb) {
            constexpr int O = decltype(O_)::value, K = decltype(K_)::value;
            constexpr int NT = (K + 7) / 8;
            const int lane = t & 31, g = lane >> 2, q = lane & 3;
            float acc[NT][4], accb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
            const uint32_t one = g == 0 ? 0x3f800000u : 0u;     // B = the ones column (n = 0): the bias gradient
#pragma unroll 2
            for (int s0 = 0; s0 < kSamples; s0 += 8) {
                // A[o][s] = D[s0 + s][o]: (g, q), (g + 8, q), (g, q + 4), (g + 8, q + 4)
                const float* d0 = row(dslot, s0 + q);
                const float* d1 = row(dslot, s0 + q + 4);
                uint32_t ah[4], al[4];
                split_tf32(d0[g], ah[0], al[0]);
                split_tf32(d0[g + 8], ah[1], al[1]);
                split_tf32(d1[g], ah[2], al[2]);
                split_tf32(d1[g + 8], ah[3], al[3]);
                const float* x0 = row(islot, s0 + q);
                const float* x1 = row(islot, s0 + q + 4);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    // B[s][k] = X[s0 + s][8 nt + k]: (q, g), (q + 4, g)
                    uint32_t bh0, bl0, bh1, bl1;
                    split_tf32(x0[8 * nt + g], bh0, bl0);
                    split_tf32(x1[8 * nt + g], bh1, bl1);
                    mma_tf32(acc[nt], al[0], al[1], al[2], al[3], bh0, bh1);
                    mma_tf32(acc[nt], ah[0], ah[1], ah[2], ah[3], bl0, bl1);
                    mma_tf32(acc[nt], ah[0], ah[1], ah[2], ah[3], bh0, bh1);
                }
                mma_tf32(accb, al[0], al[1], al[2], al[3], one, one);
                mma_tf32(accb, ah[0], ah[1], ah[2], ah[3], one, one);
            }
            // D[o][k] fragments: (g, 2q), (g, 2q + 1), (g + 8, 2q), (g + 8, 2q + 1)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int o = g + (i >= 2 ? 8 : 0), k = 8 * nt + 2 * q + (i & 1);
                    if (o < O && k < K) out[bW + o * K + k] = acc[nt][i];
                }
            if (q == 0) {
                if (g < O) out[bb + g] = accb[0];
                if (g + 8 < O) out[bb + g + 8] = accb[2];
            }
        };
        if constexpr (!kBF16) {
            // six layers over the block's four warps: E1 + D2, E2 + D3, E3, D1
            const int warp = t >> 5;
            if (warp == 0) {
                mma_grad(W_{}, IE{}, S::DA1E, S::IN1E, S::E1, S::e1);
                mma_grad(W_{}, W_{}, S::DA2D, S::H1D, S::D2, S::d2);
            } else if (warp == 1) {
                mma_grad(W_{}, W_{}, S::DA2E, S::H1E, S::E2, S::e2);
                mma_grad(P2{}, W_{}, S::DY, S::H2D, S::D3, S::d3);
            } else if (warp == 2) {
                mma_grad(L2{}, W_{}, S::DOE, S::H2E, S::E3, S::e3);
            } else {
                mma_grad(W_{}, ID{}, S::DA1D, S::IN1D, S::D1, S::d1);
            }
        } else {
            for (int it = t; it < B6; it += kSamples) {
                if (it < B1) tiles(W_{}, IE{}, S::DA1E, S::IN1E, S::E1, S::e1, it);
                else if (it < B2) tiles(W_{}, W_{}, S::DA2E, S::H1E, S::E2, S::e2, it - B1);
                else if (it < B3) tiles(L2{}, W_{}, S::DOE, S::H2E, S::E3, S::e3, it - B2);
                else if (it < B4) tiles(W_{}, ID{}, S::DA1D, S::IN1D, S::D1, S::d1, it - B3);
                else if (it < B5) tiles(W_{}, W_{}, S::DA2D, S::H1D, S::D2, S::d2, it - B4);
                else tiles(P2{}, W_{}, S::DY, S::H2D, S::D3, S::d3, it - B5);
            }
        }
    }
    if (t == 0) {
        float r = 0.0f, k = 0.0f;
        for (int w = 0; w < kSamples / 32; ++w) { r += s_rec[w]; k += s_kl[w]; }
        out[S::NP] = r;
        out[S::NP + 1] = k;
    }
}

// grad[p] = sum over blocks of partial[blk][p]; loss3 = (rec + kl, rec, kl) / B.  Entries from p_begin on (np
// for the loss terms alone).  A block handles 32 consecutive
// entries (one per lane); its warp w adds rows w, w + 8, w + 16, ... in that order, and the eight warp sums are
// then added in warp order, so the result does not depend on scheduling (bit-reproducible).
constexpr int kReduceWarps = 8;

__global__ void __launch_bounds__(32 * kReduceWarps) reduce_partials(const float* __restrict__ partial, int nblk,
                                                                     int np, uint64_t B, float* __restrict__ grad,
                                                                     float* __restrict__ loss3, int p_begin)
{
    __shared__ float s_sum[kReduceWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = p_begin + blockIdx.x * 32 + lane;
    float acc = 0.0f;
    if (p < np + 2) {
#pragma unroll 8
        for (int blk = w; blk < nblk; blk += kReduceWarps) acc += __ldg(partial + (size_t)blk * (np + 2) + p);
    }
    s_sum[w][lane] = acc;
    __syncthreads();
    if (w != 0 || p >= np + 2) return;
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < kReduceWarps; ++k) t += s_sum[k][lane];
    if (p < np) {
        if (grad) grad[p] = t;
    } else if (loss3) {
        const float v = t / (float)B;
        if (p == np) { loss3[1] = v; } else { loss3[2] = v; }
    }
}

__global__ void finish_loss(float* loss3)
{
    if (threadIdx.x == 0 && loss3) loss3[0] = loss3[1] + loss3[2];
}

__global__ void adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                     const float* __restrict__ g, uint64_t n, float lr, float b1, float b2, float eps, float wd,
                     float c1, float c2)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float w = p[i];
    if (wd != 0.0f) w = w - lr * wd * w;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] = w - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---- graph-replayable step: everything keyed by a step counter in device memory ----

// Mini-batch b of step t: record index mulhi(w, n) with w word 0 of counter (t, b, 0, 0xB0) (uniform, with
// replacement), and the latent normals of counter (0, b, t, 0xE0) (the same as the host-step path).
__global__ void gather_batch(const float* __restrict__ x_all, const float* __restrict__ c_all, uint64_t n, int p_out,
                             int p_in, int latent, uint64_t B, uint64_t seed,
                             const unsigned long long* __restrict__ step, float* __restrict__ xb,
                             float* __restrict__ cb, float* __restrict__ eps)
{
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const unsigned long long t = *step;
    const Stream pick(seed, ((uint64_t)(uint32_t)t) | (b << 32));
    const Words w = pick.at((uint32_t)(t >> 32), 0xB0u);
    const uint64_t i = ((uint64_t)w.w0 * n) >> 32;
    for (int j = 0; j < p_out; ++j) xb[b * p_out + j] = x_all[i * p_out + j];
    for (int j = 0; j < p_in; ++j) cb[b * p_in + j] = c_all[i * p_in + j];
    const Stream st(seed, (t << 32) | (b & 0xffffffffull));
    for (int j = 0; 4 * j < latent; ++j) {
        const Words e = st.at((uint32_t)j, 0xE0u);
        const float2 p0 = box_muller(e.w0, e.w1), p1 = box_muller(e.w2, e.w3);
        const float v[4] = {p0.x, p0.y, p1.x, p1.y};
        for (int i = 0; i < 4 && 4 * j + i < latent; ++i) eps[b * latent + 4 * j + i] = v[i];
    }
}

// Adam with the step t read from device memory (bias corrections computed here).
__global__ void adam_dev(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                         const float* __restrict__ g, uint64_t n, float lr, float b1, float b2, float eps, float wd,
                         const unsigned long long* __restrict__ step)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double t = (double)*step;
    const float c1 = (float)(1.0 - pow((double)b1, t));
    const float c2 = (float)(1.0 - pow((double)b2, t));
    float w = p[i];
    if (wd != 0.0f) w = w - lr * wd * w;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] = w - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void bump_step(unsigned long long* step)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1ull;
}

using LaunchFn = cudaError_t (*)(const float*, const float*, const float*, const float*, uint64_t, uint64_t, uint64_t,
                                 float*, cudaStream_t);
struct Plan {
    int np = 0;
    LaunchFn launch = nullptr;       // forward and backward
    LaunchFn launch_fwd = nullptr;   // the loss alone
};

template <int PI, int PO, int W, int L, bool kBF16, bool kGrad>
cudaError_t launch_fb(const float* prm, const float* X, const float* C, const float* E, uint64_t B, uint64_t seed,
                      uint64_t step, float* partial, cudaStream_t s)
{
    using S = Shape<PI, PO, W, L>;
    const size_t smem = ((kGrad ? (size_t)S::NSLOT * S::SLOT : 0) + S::SW) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(fwd_bwd<PI, PO, W, L, kBF16, kGrad>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned nblk = (unsigned)((B + kSamples - 1) / kSamples);
    fwd_bwd<PI, PO, W, L, kBF16, kGrad><<<nblk, kSamples, smem, s>>>(prm, X, C, E, B, seed, step, partial);
    return cudaGetLastError();
}

// Compiled shapes (p_in, p_out, width, latent): the uniform width-16 / latent-4 set, and the final Table 1
// shapes of LengthGen, PathGen and EventGen.
#define MS_TRAIN_SHAPES(X)                                                                                    \
    X(1, 1, 16, 4) X(2, 1, 16, 4) X(3, 3, 16, 4) X(4, 1, 16, 4) X(4, 3, 16, 4) X(4, 6, 16, 4) X(7, 6, 16, 4)   \
    X(2, 1, 8, 2) X(3, 3, 16, 5) X(7, 6, 16, 5)

Plan plan_for(const ms_cvae_shape& sh)
{
    Plan pl;
#define MS_CASE(pi, po, w, l)                                                                                  \
    if (sh.p_in == pi && sh.p_out == po && sh.width == w && sh.latent == l) {                                 \
        pl.np = Shape<pi, po, w, l>::NP;                                                                      \
        pl.launch = sh.precision == MS_BF16 ? launch_fb<pi, po, w, l, true, true>                             \
                                            : launch_fb<pi, po, w, l, false, true>;                           \
        pl.launch_fwd = sh.precision == MS_BF16 ? launch_fb<pi, po, w, l, true, false>                        \
                                                : launch_fb<pi, po, w, l, false, false>;                      \
    }
    MS_TRAIN_SHAPES(MS_CASE)
#undef MS_CASE
    return pl;
}

}  // namespace train
}  // namespace ms

using namespace ms::train;

extern "C" size_t ms_cvae_num_params(const ms_cvae_shape* s)
{
    if (!s) return 0;
    const size_t W = (size_t)s->width, L = (size_t)s->latent, PI = (size_t)s->p_in, PO = (size_t)s->p_out;
    const size_t enc = W * (PO + PI) + W + W * W + W + 2 * L * W + 2 * L;
    const size_t dec = W * (PI + L) + W + W * W + W + 2 * PO * W + 2 * PO;
    return enc + dec;
}

extern "C" size_t ms_cvae_workspace_size(const ms_cvae_shape* s, uint64_t batch)
{
    if (!s) return 0;
    const size_t nblk = (size_t)((batch + kSamples - 1) / kSamples);
    const size_t np = ms_cvae_num_params(s);
    const size_t partial = nblk * (np + 2) * sizeof(float);
    const size_t grad = np * sizeof(float);
    return ((partial + 255) & ~(size_t)255) + ((grad + 255) & ~(size_t)255);
}

static ms_status check_shape(const ms_cvae_shape* s, const char* fn, Plan* out)
{
    if (!s) return ms::set_error(MS_ERR_INVALID_ARG, "%s: null shape", fn);
    if (s->precision != MS_FP32 && s->precision != MS_BF16)
        return ms::set_error(MS_ERR_UNSUPPORTED, "%s: training precision must be MS_FP32 or MS_BF16", fn);
    *out = plan_for(*s);
    if (!out->launch)
        return ms::set_error(MS_ERR_UNSUPPORTED,
                             "%s: shape (p_in %d, p_out %d, latent %d, width %d) is not built; built: latent 4, "
                             "width 16, (p_in, p_out) in (1,1) (2,1) (3,3) (4,1) (4,3) (4,6) (7,6); and "
                             "(2,1) latent 2 width 8, (3,3) and (7,6) latent 5 width 16",
                             fn, s->p_in, s->p_out, s->latent, s->width);
    return MS_OK;
}

extern "C" ms_status ms_cvae_forward_backward(const ms_cvae_shape* s, const float* params, const float* x,
                                              const float* c, const float* eps_z, uint64_t B, uint64_t seed,
                                              uint64_t step, float* grad, float* loss3, void* workspace,
                                              size_t workspace_bytes, void* stream)
{
    MS_NVTX("ms_cvae_forward_backward");
    Plan pl;
    ms_status st = check_shape(s, "ms_cvae_forward_backward", &pl);
    if (st != MS_OK) return st;
    MS_CHECK_ARG(B >= 1 && B < (1ull << 32), "ms_cvae_forward_backward: batch must be in [1, 2^32)");
    MS_CHECK_ARG(params && x && c, "ms_cvae_forward_backward: null params, x or c");
    MS_CHECK_ARG(workspace && workspace_bytes >= ms_cvae_workspace_size(s, B),
                 "ms_cvae_forward_backward: workspace of at least %zu bytes required", ms_cvae_workspace_size(s, B));
    MS_CHECK_ARG(((uintptr_t)workspace & 255u) == 0, "ms_cvae_forward_backward: workspace must be 256-byte aligned");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    float* partial = static_cast<float*>(workspace);
    const int nblk = (int)((B + kSamples - 1) / kSamples);
    MS_CUDA(pl.launch(params, x, c, eps_z, B, seed, step, partial, cs));
    const int n = pl.np + 2;
    reduce_partials<<<(n + 31) / 32, 32 * kReduceWarps, 0, cs>>>(partial, nblk, pl.np, B, grad, loss3, 0);
    MS_CUDA(cudaGetLastError());
    finish_loss<<<1, 32, 0, cs>>>(loss3);
    MS_CUDA(cudaGetLastError());
    return MS_OK;
}

extern "C" ms_status ms_cvae_forward(const ms_cvae_shape* s, const float* params, const float* x, const float* c,
                                     const float* eps_z, uint64_t B, uint64_t seed, uint64_t step, float* loss3,
                                     void* workspace, size_t workspace_bytes, void* stream)
{
    MS_NVTX("ms_cvae_forward");
    Plan pl;
    ms_status st = check_shape(s, "ms_cvae_forward", &pl);
    if (st != MS_OK) return st;
    MS_CHECK_ARG(B >= 1 && B < (1ull << 32), "ms_cvae_forward: batch must be in [1, 2^32)");
    MS_CHECK_ARG(params && x && c && loss3, "ms_cvae_forward: null params, x, c or loss3");
    MS_CHECK_ARG(workspace && workspace_bytes >= ms_cvae_workspace_size(s, B),
                 "ms_cvae_forward: workspace of at least %zu bytes required", ms_cvae_workspace_size(s, B));
    MS_CHECK_ARG(((uintptr_t)workspace & 255u) == 0, "ms_cvae_forward: workspace must be 256-byte aligned");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    float* partial = static_cast<float*>(workspace);
    const int nblk = (int)((B + kSamples - 1) / kSamples);
    MS_CUDA(pl.launch_fwd(params, x, c, eps_z, B, seed, step, partial, cs));
    reduce_partials<<<1, 32 * kReduceWarps, 0, cs>>>(partial, nblk, pl.np, B, nullptr, loss3, pl.np);
    MS_CUDA(cudaGetLastError());
    finish_loss<<<1, 32, 0, cs>>>(loss3);
    MS_CUDA(cudaGetLastError());
    return MS_OK;
}

extern "C" ms_status ms_adam_step(float* params, float* m, float* v, const float* grad, uint64_t n, uint64_t t,
                                  float lr, float beta1, float beta2, float eps, float weight_decay, void* stream)
{
    MS_NVTX("ms_adam_step");
    MS_CHECK_ARG(params && m && v && grad, "ms_adam_step: null array");
    MS_CHECK_ARG(t >= 1, "ms_adam_step: step t must be >= 1");
    if (n == 0) return MS_OK;
    const float c1 = (float)(1.0 - std::pow((double)beta1, (double)t));
    const float c2 = (float)(1.0 - std::pow((double)beta2, (double)t));
    adam<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(params, m, v, grad, n, lr, beta1,
                                                                                    beta2, eps, weight_decay, c1, c2);
    MS_CUDA(cudaGetLastError());
    return MS_OK;
}

extern "C" ms_status ms_cvae_train_step(const ms_cvae_shape* s, float* params, float* m, float* v, const float* x,
                                        const float* c, const float* eps_z, uint64_t B, uint64_t seed, uint64_t step,
                                        float lr, float weight_decay, float* loss3, void* workspace,
                                        size_t workspace_bytes, void* stream)
{
    MS_NVTX("ms_cvae_train_step");
    Plan pl;
    ms_status st = check_shape(s, "ms_cvae_train_step", &pl);
    if (st != MS_OK) return st;
    MS_CHECK_ARG(step >= 1, "ms_cvae_train_step: step must be >= 1");
    MS_CHECK_ARG(B >= 1 && B < (1ull << 32), "ms_cvae_train_step: batch must be in [1, 2^32)");
    MS_CHECK_ARG(workspace && workspace_bytes >= ms_cvae_workspace_size(s, B),
                 "ms_cvae_train_step: workspace of at least %zu bytes required", ms_cvae_workspace_size(s, B));
    const size_t nblk = (size_t)((B + kSamples - 1) / kSamples);
    const size_t partial_bytes = ((nblk * (pl.np + 2) * sizeof(float)) + 255) & ~(size_t)255;
    float* grad = reinterpret_cast<float*>(static_cast<char*>(workspace) + partial_bytes);
    st = ms_cvae_forward_backward(s, params, x, c, eps_z, B, seed, step, grad, loss3, workspace, workspace_bytes,
                                  stream);
    if (st != MS_OK) return st;
    return ms_adam_step(params, m, v, grad, (uint64_t)pl.np, step, lr, 0.9f, 0.999f, 1e-8f, weight_decay, stream);
}

// Scratch of the device-step training step: the ms_cvae_train_step workspace, then the gathered batch and its
// latent normals.
static size_t dev_step_extra(const ms_cvae_shape* s, uint64_t B)
{
    const size_t f = (size_t)B * (size_t)(s->p_out + s->p_in + s->latent) * sizeof(float);
    return (f + 255) & ~(size_t)255;
}

extern "C" size_t ms_cvae_train_step_dev_workspace_size(const ms_cvae_shape* s, uint64_t batch)
{
    if (!s) return 0;
    return ms_cvae_workspace_size(s, batch) + dev_step_extra(s, batch);
}

extern "C" ms_status ms_cvae_train_step_dev(const ms_cvae_shape* s, float* params, float* m, float* v,
                                            const float* x_all, const float* c_all, uint64_t n_records, uint64_t B,
                                            uint64_t seed, unsigned long long* step, float lr, float weight_decay,
                                            float* loss3, void* workspace, size_t workspace_bytes, void* stream)
{
    MS_NVTX("ms_cvae_train_step_dev");
    Plan pl;
    ms_status st = check_shape(s, "ms_cvae_train_step_dev", &pl);
    if (st != MS_OK) return st;
    MS_CHECK_ARG(x_all && c_all && step && params && m && v, "ms_cvae_train_step_dev: null argument");
    MS_CHECK_ARG(n_records >= 1 && n_records < (1ull << 32), "ms_cvae_train_step_dev: 1 <= n_records < 2^32");
    MS_CHECK_ARG(B >= 1 && B < (1ull << 31), "ms_cvae_train_step_dev: batch must be in [1, 2^31)");
    const size_t base = ms_cvae_workspace_size(s, B);
    MS_CHECK_ARG(workspace && workspace_bytes >= base + dev_step_extra(s, B) && ((uintptr_t)workspace & 255u) == 0,
                 "ms_cvae_train_step_dev: a 256-byte aligned workspace of ms_cvae_train_step_dev_workspace_size() "
                 "bytes is required");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    float* xb = reinterpret_cast<float*>(static_cast<char*>(workspace) + base);
    float* cb = xb + B * s->p_out;
    float* eps = cb + B * s->p_in;
    gather_batch<<<(unsigned)((B + 255) / 256), 256, 0, cs>>>(x_all, c_all, n_records, s->p_out, s->p_in, s->latent,
                                                                B, seed, step, xb, cb, eps);
    MS_CUDA(cudaGetLastError());
    const size_t nblk = (size_t)((B + kSamples - 1) / kSamples);
    const size_t partial_bytes = ((nblk * (pl.np + 2) * sizeof(float)) + 255) & ~(size_t)255;
    float* grad = reinterpret_cast<float*>(static_cast<char*>(workspace) + partial_bytes);
    st = ms_cvae_forward_backward(s, params, xb, cb, eps, B, seed, 0, grad, loss3, workspace, base, stream);
    if (st != MS_OK) return st;
    adam_dev<<<(unsigned)((pl.np + 255) / 256), 256, 0, cs>>>(params, m, v, grad, (uint64_t)pl.np, lr, 0.9f, 0.999f,
                                                               1e-8f, weight_decay, step);
    MS_CUDA(cudaGetLastError());
    bump_step<<<1, 32, 0, cs>>>(step);
    MS_CUDA(cudaGetLastError());
    return MS_OK;
}
