// Device building blocks shared by the library's kernels: the counter-based generator, uniform and normal
// draws, and the host-side status plumbing.  Written for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ms.h"

namespace ms {

// ---------------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 multiplications with the
// round multipliers on counter words 0 and 2, XOR of the high halves with the opposite words and the round
// key, and a word permutation; the key advances by the two Weyl constants between rounds.
// Counter layout used throughout the library: (step, id_lo, id_hi, tag), key = (seed_lo, seed_hi).
struct Words { uint32_t w0, w1, w2, w3; };

__device__ __forceinline__ Words philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1)
{
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hiA = __umulhi(kMulA, c0), loA = kMulA * c0;
        const uint32_t hiB = __umulhi(kMulB, c2), loB = kMulB * c2;
        const uint32_t n0 = hiB ^ c1 ^ k0, n2 = hiA ^ c3 ^ k1;
        c0 = n0; c1 = loB; c2 = n2; c3 = loA;
        k0 += kWeylA; k1 += kWeylB;
    }
    return Words{c0, c1, c2, c3};
}

struct Stream {
    uint32_t k0, k1, id_lo, id_hi;
    __device__ __forceinline__ Stream(uint64_t seed, uint64_t id)
        : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), id_lo((uint32_t)id), id_hi((uint32_t)(id >> 32)) {}
    __device__ __forceinline__ Words at(uint32_t step, uint32_t tag) const
    {
        return philox(step, id_lo, id_hi, tag, k0, k1);
    }
};

// 24-bit uniform in [0, 1): exact in single precision.
__device__ __forceinline__ float u24(uint32_t w) { return (float)(w >> 8) * 0x1.0p-24f; }

// 53-bit uniform in [0, 1) from a high and a low word.
__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo)
{
    return (double)(((uint64_t)hi << 21) | (uint64_t)(lo >> 11)) * 0x1.0p-53;
}

// sin and cos of 2*pi*u for u in [0, 1): shift the angle into [-pi, pi) where the hardware approximations are
// accurate, then undo the half-turn by a sign flip.
__device__ __forceinline__ void sincos_turns_fast(float u, float* s, float* c)
{
    float sn, cs;
    __sincosf(6.28318530717958647692f * (u - 0.5f), &sn, &cs);
    *s = -sn;
    *c = -cs;
}

// Square root on the special-function unit's approximation (relative error about 2^-23; no IEEE rounding and
// none of the correctly rounded square root's special-case branch).
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Box-Muller: two standard normals from two 24-bit uniforms.
__device__ __forceinline__ float2 box_muller(uint32_t wa, uint32_t wb)
{
    const float r = sqrt_approx(-2.0f * __logf(1.0f - u24(wa)));
    float s, c;
    sincos_turns_fast(u24(wb), &s, &c);
    return make_float2(r * c, r * s);
}

__device__ __forceinline__ float softplus(float x)
{
    return fmaxf(x, 0.0f) + __logf(1.0f + __expf(-fabsf(x)));
}

// Warp-aggregated ticket: every lane with `want` set receives a distinct index from *counter.
__device__ __forceinline__ unsigned long long warp_ticket(unsigned long long* counter, bool want)
{
    const unsigned mask = __ballot_sync(0xffffffffu, want);
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    const int leader = mask ? __ffs(mask) - 1 : 0;
    if (mask && lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + (unsigned long long)__popc(mask & ((1u << lane) - 1u));
}

}  // namespace ms

// ---------------------------------------------------------------------------------------------------------
// Tracing: every compute entry point of the C ABI opens an NVTX range named after itself for its duration on the
// host (what it validates and enqueues), so profilers can attribute launches to ABI calls (for example
// `ncu --nvtx --nvtx-include "ms_render/"`).  NVTX is header-only: without a profiler attached the range calls
// return at once.
#include <nvtx3/nvToolsExt.h>
namespace ms {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace ms
#define MS_NVTX(name) ::ms::NvtxRange ms_nvtx_range_(name)

// ---------------------------------------------------------------------------------------------------------
// Host-side status plumbing (defined in capi.cu).
namespace ms {
ms_status set_error(ms_status st, const char* fmt, ...);
ms_status cuda_status(cudaError_t e, const char* what);
int num_sms();
}  // namespace ms

#define MS_CHECK_ARG(cond, ...)                                                                            \
    do {                                                                                                   \
        if (!(cond)) return ::ms::set_error(MS_ERR_INVALID_ARG, __VA_ARGS__);                              \
    } while (0)

#define MS_CUDA(expr)                                                                                      \
    do {                                                                                                   \
        cudaError_t e_ = (expr);                                                                           \
        if (e_ != cudaSuccess) return ::ms::cuda_status(e_, #expr);                                        \
    } while (0)
