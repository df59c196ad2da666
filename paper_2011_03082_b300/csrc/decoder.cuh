// The query's standard normals for the CVAE decoder sampling (Sec. 3.2).
#pragma once

#include "ms_device.cuh"

namespace ms {
namespace dec {

// Standard normals 4j..4j+3 of a query: counter (j, id_lo, id_hi, tag), Box-Muller on word pairs.
__device__ __forceinline__ float4 normals4(const Stream& st, uint32_t j, uint32_t tag)
{
    const Words w = st.at(j, tag);
    const float2 a = box_muller(w.w0, w.w1), b = box_muller(w.w2, w.w3);
    return make_float4(a.x, a.y, b.x, b.y);
}

}  // namespace dec
}  // namespace ms
