// ms_training_records: walk records -> the three CVAEs' conditions and targets (Sec. 4.1, Eq. 3; Eq. 4 read
// backwards).  One thread per record; memory bound (about 90 bytes read and 88 written per record).
#include "ms_device.cuh"

namespace ms {
namespace rec {

__global__ void records_kernel(uint64_t n, const int32_t* __restrict__ n_events, const float* __restrict__ xp,
                               const float* __restrict__ wp, const float* __restrict__ Xp,
                               const float* __restrict__ Wp, const ms_medium* __restrict__ media, int per,
                               uint64_t seed, float* __restrict__ cL, float* __restrict__ xL, float* __restrict__ cP,
                               float* __restrict__ xP, float* __restrict__ cE, float* __restrict__ xE)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x0 = xp[3 * i], x1 = xp[3 * i + 1], x2 = xp[3 * i + 2];
    // rotation about (0,0,1) by -psi, psi = atan2(x_y, x_x): cos psi = x_x / rho, sin psi = x_y / rho
    const float rho = sqrtf(x0 * x0 + x1 * x1);
    const float cs = rho > 0.0f ? x0 / rho : 1.0f, sn = rho > 0.0f ? x1 / rho : 0.0f;
    auto rx = [&](float a, float b) { return cs * a + sn * b; };
    auto ry = [&](float a, float b) { return -sn * a + cs * b; };
    const float w0 = wp[3 * i], w1 = wp[3 * i + 1], w2 = wp[3 * i + 2];
    const float ct = x2;
    const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    const float wr0 = rx(w0, w1), wr1 = ry(w0, w1);
    const float alpha = wr1;
    const float beta = wr0 * ct - w2 * st;
    const ms_medium m = media[per ? i : 0];
    const float ltau = logf(m.optical_radius);
    const int32_t N = n_events[i];
    const float lnN = logf((float)N);
    const Stream s(seed, i);
    const float u = u24(s.at(0u, 0x44u).w0);
    const float yN = logf((float)N - 0.5f + u);
    cL[2 * i] = ltau; cL[2 * i + 1] = m.g;
    xL[i] = yN;
    cP[3 * i] = ltau; cP[3 * i + 1] = m.g; cP[3 * i + 2] = lnN;
    xP[3 * i] = ct; xP[3 * i + 1] = alpha; xP[3 * i + 2] = beta;
    float* ce = cE + 7 * i;
    ce[0] = ltau; ce[1] = m.g; ce[2] = m.albedo; ce[3] = ct; ce[4] = alpha; ce[5] = beta; ce[6] = lnN;
    const float X0 = Xp[3 * i], X1 = Xp[3 * i + 1], X2 = Xp[3 * i + 2];
    const float V0 = Wp[3 * i], V1 = Wp[3 * i + 1], V2 = Wp[3 * i + 2];
    float* xe = xE + 6 * i;
    xe[0] = rx(X0, X1); xe[1] = ry(X0, X1); xe[2] = X2;
    xe[3] = rx(V0, V1); xe[4] = ry(V0, V1); xe[5] = V2;
}

}  // namespace rec
}  // namespace ms

extern "C" ms_status ms_training_records(uint64_t n, const int32_t* n_events, const float* exit_pos,
                                         const float* exit_dir, const float* rep_pos, const float* rep_dir,
                                         const ms_medium* media, int32_t per_photon_media, uint64_t seed, float* cL,
                                         float* xL, float* cP, float* xP, float* cE, float* xE, void* stream)
{
    MS_NVTX("ms_training_records");
    MS_CHECK_ARG(n_events && exit_pos && exit_dir && rep_pos && rep_dir && media,
                 "ms_training_records: null input");
    MS_CHECK_ARG(cL && xL && cP && xP && cE && xE, "ms_training_records: null output");
    if (n == 0) return MS_OK;
    const unsigned grid = (unsigned)((n + 255) / 256);
    ms::rec::records_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, n_events, exit_pos, exit_dir, rep_pos, rep_dir, media, per_photon_media, seed, cL, xL, cP, xP, cE, xE);
    MS_CUDA(cudaGetLastError());
    return MS_OK;
}
