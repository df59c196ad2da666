// The query's standard normals for the CVAE decoder sampling (Sec. 3.2).
#pragma once

#include "ms_device.cuh"

namespace ms {
namespace dec {

// The count standard normals of a query come from the fewest Philox blocks B (counters (j, id_lo, id_hi, tag),
// j < B) whose 4B words give the 2 ceil(count / 2) uniforms that Box-Muller needs: uniform k < 4B is the top 24
// bits of word k (block k / 4, word k % 4), and uniform 4B + i is the low bytes of words 3i, 3i+1, 3i+2 (which
// the top bits leave unused), so B blocks give 4B + floor(4B / 3) uniforms.  Normals 2m, 2m+1 are Box-Muller on
// uniforms 2m, 2m+1.  (Ten normals take two blocks instead of three.)
__host__ __device__ constexpr int normal_blocks(int count)
{
    int b = 1;
    while (4 * b + (4 * b) / 3 < count + (count & 1)) ++b;
    return b;
}

__device__ __forceinline__ uint32_t spare_uniform_word(uint32_t a, uint32_t b, uint32_t c)
{
    // a 24-bit word in the top bits, as u24 expects
    return (((a & 0xffu) << 16) | ((b & 0xffu) << 8) | (c & 0xffu)) << 8;
}

// The first NZ normals of a query into out[0 .. NZ) (compile-time count; everything stays in registers).
template <int NZ, int N>
__device__ __forceinline__ void query_normals_philox(const Stream& st, uint32_t tag, float (&out)[N])
{
    static_assert(N >= NZ, "output row too short");
    constexpr int kB = normal_blocks(NZ);
    constexpr int kPairs = (NZ + 1) / 2;
    uint32_t w[4 * kB];
#pragma unroll
    for (int j = 0; j < kB; ++j) {
        const Words v = st.at((uint32_t)j, tag);
        w[4 * j] = v.w0; w[4 * j + 1] = v.w1; w[4 * j + 2] = v.w2; w[4 * j + 3] = v.w3;
    }
#pragma unroll
    for (int m = 0; m < kPairs; ++m) {
        const int ka = 2 * m, kb = 2 * m + 1, ia = ka - 4 * kB, ib = kb - 4 * kB;
        const uint32_t wa = ka < 4 * kB ? w[ka] : spare_uniform_word(w[3 * ia], w[3 * ia + 1], w[3 * ia + 2]);
        const uint32_t wb = kb < 4 * kB ? w[kb] : spare_uniform_word(w[3 * ib], w[3 * ib + 1], w[3 * ib + 2]);
        const float2 z = box_muller(wa, wb);
        out[2 * m] = z.x;
        if (2 * m + 1 < NZ) out[2 * m + 1] = z.y;
    }
}

// The first count (<= 16) normals of a query into out[0 .. count), for runtime counts.
__device__ __forceinline__ void query_normals_runtime(const Stream& st, uint32_t tag, int count, float* out)
{
    const int nb = normal_blocks(count);       // <= 3 for 16 normals
    uint32_t w[12];
    for (int j = 0; j < nb; ++j) {
        const Words v = st.at((uint32_t)j, tag);
        w[4 * j] = v.w0; w[4 * j + 1] = v.w1; w[4 * j + 2] = v.w2; w[4 * j + 3] = v.w3;
    }
    auto uw = [&](int k) -> uint32_t {
        if (k < 4 * nb) return w[k];
        const int i = k - 4 * nb;
        return spare_uniform_word(w[3 * i], w[3 * i + 1], w[3 * i + 2]);
    };
    for (int m = 0; 2 * m < count; ++m) {
        const float2 z = box_muller(uw(2 * m), uw(2 * m + 1));
        out[2 * m] = z.x;
        if (2 * m + 1 < count) out[2 * m + 1] = z.y;
    }
}

}  // namespace dec
}  // namespace ms
