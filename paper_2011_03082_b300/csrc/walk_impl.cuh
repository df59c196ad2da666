// Brute-force Henyey-Greenstein random walk in the unit sphere (Sec. 3.1, Eq. 1) with the representative
// event reservoir of Sec. 4.3 — the plain method, the renderer's thin-region fallback and the generator of
// the models' training data.
//
// Kernel design (one B300, 148 SMs):
//  * persistent grid, one lane per photon in flight; a lane that finishes refills at once from its warp's
//    chunk of photon ids, and the warp fetches a new chunk of 32 ids from a global ticket with one atomic,
//    so warps stay full although path lengths differ by orders of magnitude;
//  * the loop body is one scattering event plus one free flight: a Philox4x32-10 block (integer pipe), a
//    log, a sin/cos pair, square roots — no memory traffic except when a photon finishes;
//  * histograms live in shared memory (integer atomics, order independent) and are added to the global
//    64-bit counters once per block, so results do not depend on the launch shape.
// The arithmetic is written once against a precision policy: `F32` (24-bit uniforms, the special-function
// unit's approximations for log, sin/cos, reciprocal and square roots) and `F64` (53-bit uniforms, the correctly rounded operations of ms_detmath.cuh in the same
// order as any other implementation of these steps; its translation unit is built without FMA contraction).
#pragma once

#include "ms_detmath.cuh"
#include "ms_device.cuh"

namespace ms {
namespace walk {

struct Job {
    uint64_t seed, offset, n;
    const ms_medium* media;
    int per_photon_media;
    uint32_t max_events;
    int reservoir;
    ms_walk_out out;
    unsigned long long* ticket;
};

constexpr int kThreads = 256;
constexpr int kChunk = 32;

struct F32 {
    using real = float;
    // u[4]: the block's four 24-bit uniforms; *ures: a fifth from the low bytes those leave unused
    static __device__ __forceinline__ void uniforms(const Stream& s, uint32_t step, uint32_t tag, real u[4],
                                                    real* ures = nullptr)
    {
        const Words w = s.at(step, tag);
        u[0] = u24(w.w0); u[1] = u24(w.w1); u[2] = u24(w.w2); u[3] = u24(w.w3);
        if (ures)
            *ures = (float)(((w.w0 & 0xffu) << 16) | ((w.w1 & 0xffu) << 8) | (w.w2 & 0xffu)) * 0x1.0p-24f;
    }
    static __device__ __forceinline__ real log(real x) { return __logf(x); }
    static __device__ __forceinline__ void sincos_turns(real u, real* s, real* c) { sincos_turns_fast(u, s, c); }
    static __device__ __forceinline__ real atan2(real y, real x) { return atan2f(y, x); }
    static __device__ __forceinline__ real sqrt(real x) { return sqrt_approx(x); }
    static __device__ __forceinline__ real div(real a, real b) { return __fdividef(a, b); }
    static __device__ __forceinline__ real inv_norm(real d) { return rsqrtf(d); }
    static constexpr bool kDivideToNormalise = false;
    static constexpr real kPi = 3.14159265358979323846f, kTwoPi = 6.28318530717958647692f;
};

struct F64 {
    using real = double;
    // u[4]: 53-bit uniforms from the tag and tag + 2 blocks; *ures: a 33-bit uniform from the low 11 bits of
    // the tag + 2 words, which those leave unused
    static __device__ __forceinline__ void uniforms(const Stream& s, uint32_t step, uint32_t tag, real u[4],
                                                    real* ures = nullptr)
    {
        const Words h = s.at(step, tag), l = s.at(step, tag + 2u);
        u[0] = u53(h.w0, l.w0); u[1] = u53(h.w1, l.w1); u[2] = u53(h.w2, l.w2); u[3] = u53(h.w3, l.w3);
        if (ures)
            *ures = (double)(((uint64_t)(l.w0 & 0x7ffu) << 22) | ((uint64_t)(l.w1 & 0x7ffu) << 11) |
                             (uint64_t)(l.w2 & 0x7ffu)) * 0x1.0p-33;
    }
    static __device__ __forceinline__ real log(real x) { return det::log(x); }
    static __device__ __forceinline__ void sincos_turns(real u, real* s, real* c) { det::sincos_turns(u, s, c); }
    static __device__ __forceinline__ real atan2(real y, real x) { return det::atan2(y, x); }
    static __device__ __forceinline__ real sqrt(real x) { return ::sqrt(x); }
    static __device__ __forceinline__ real div(real a, real b) { return a / b; }
    static __device__ __forceinline__ real inv_norm(real d) { return 1.0 / ::sqrt(d); }
    static constexpr bool kDivideToNormalise = true;
    static constexpr real kPi = det::kPi, kTwoPi = det::kTwoPi;
};

template <class Pol>
struct V3 {
    typename Pol::real x, y, z;
};

template <class Pol>
__device__ __forceinline__ typename Pol::real dot(const V3<Pol>& a, const V3<Pol>& b)
{
    return a.x * b.x + a.y * b.y + a.z * b.z;
}

template <class Pol>
__device__ __forceinline__ V3<Pol> unit(V3<Pol> v)
{
    using real = typename Pol::real;
    const real d = dot<Pol>(v, v);
    if (Pol::kDivideToNormalise) {
        const real n = Pol::sqrt(d);
        v.x = v.x / n; v.y = v.y / n; v.z = v.z / n;
    } else {
        const real s = Pol::inv_norm(d);
        v.x = v.x * s; v.y = v.y * s; v.z = v.z * s;
    }
    return v;
}

// Inverse CDF of the HG phase function (Eq. 1): cosine between the old and the new propagation direction.
template <class Pol>
__device__ __forceinline__ typename Pol::real hg_cosine(typename Pol::real u, typename Pol::real g)
{
    using real = typename Pol::real;
    if (fabs(g) < (real)1e-4) return (real)2 * u - (real)1;
    const real t = Pol::div((real)1 - g * g, (real)1 - g + (real)2 * g * u);
    real mu = Pol::div((real)1 + g * g - t * t, (real)2 * g);
    mu = mu < (real)-1 ? (real)-1 : mu;
    mu = mu > (real)1 ? (real)1 : mu;
    return mu;
}

// New direction at polar cosine mu and azimuth 2 pi u around w, in the orthonormal basis of Duff et al.
// (JCGT 2017), renormalised.
template <class Pol>
__device__ __forceinline__ V3<Pol> scatter(const V3<Pol>& w, typename Pol::real mu, typename Pol::real u)
{
    using real = typename Pol::real;
    const real sign = w.z >= (real)0 ? (real)1 : (real)-1;
    const real a = Pol::div((real)-1, sign + w.z);
    const real b = w.x * w.y * a;
    const V3<Pol> t1{(real)1 + sign * w.x * w.x * a, sign * b, -sign * w.x};
    const V3<Pol> t2{b, sign + w.y * w.y * a, -w.y};
    const real one_m = (real)1 - mu * mu;
    const real st = Pol::sqrt(one_m > (real)0 ? one_m : (real)0);
    real sp, cp;
    Pol::sincos_turns(u, &sp, &cp);
    const real ca = st * cp, sa = st * sp;
    V3<Pol> r{ca * t1.x + sa * t2.x + mu * w.x, ca * t1.y + sa * t2.y + mu * w.y, ca * t1.z + sa * t2.z + mu * w.z};
    return unit<Pol>(r);
}

template <class Pol>
__device__ __forceinline__ V3<Pol> isotropic(typename Pol::real uz, typename Pol::real uphi)
{
    using real = typename Pol::real;
    const real z = (real)1 - (real)2 * uz;
    const real one_m = (real)1 - z * z;
    const real st = Pol::sqrt(one_m > (real)0 ? one_m : (real)0);
    real sp, cp;
    Pol::sincos_turns(uphi, &sp, &cp);
    return V3<Pol>{st * cp, st * sp, z};
}

__device__ __forceinline__ int hist_n_bin(uint32_t n)
{
    if (n == 0) return 0;
    const int e = 31 - __clz(n);
    const int m = (int)((((uint64_t)n << 2) >> e) & 3u);
    const int b = 1 + 4 * e + m;
    return b > 63 ? 63 : b;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <class Pol>
struct Photon {
    using real = typename Pol::real;
    uint64_t i;                 // local index (id - offset)
    V3<Pol> p, w, rep_p, rep_w;
    real sig, g, phi, pw, wsum;
    uint32_t n, step;
    int32_t rep_k;
    bool paper;
};

template <class Pol>
__global__ void __launch_bounds__(kThreads) walk_kernel(Job J)
{
    using real = typename Pol::real;
    __shared__ unsigned s_hist_n[64], s_hist_cos[64], s_hist_pos[32 * 64];
    __shared__ unsigned long long s_cnt[4];
    for (int k = threadIdx.x; k < 32 * 64; k += kThreads) s_hist_pos[k] = 0u;
    if (threadIdx.x < 64) { s_hist_n[threadIdx.x] = 0u; s_hist_cos[threadIdx.x] = 0u; }
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0ull;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    const uint32_t key_lo = (uint32_t)J.seed, key_hi = (uint32_t)(J.seed >> 32);
    (void)key_lo; (void)key_hi;

    Photon<Pol> ph;
    bool active = false;
    unsigned long long my_escaped = 0, my_absorbed = 0, my_truncated = 0, my_events = 0;
    uint64_t next = 0, end = 0;   // warp-uniform chunk of photon indices
    bool drained = false;         // warp-uniform: the global ticket is exhausted

    for (;;) {
        // ---- refill idle lanes from the warp's chunk (warp-uniform control flow) ----
        unsigned need = __ballot_sync(0xffffffffu, !active);
        while (need && !drained) {
            if (next >= end) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(J.ticket, (unsigned long long)kChunk);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= J.n) { drained = true; break; }
                next = base;
                end = base + kChunk < J.n ? base + kChunk : J.n;
            }
            const unsigned avail = (unsigned)(end - next);
            const unsigned rank = __popc(need & lanemask_lt);
            const bool mine = ((need >> lane) & 1u) && rank < avail;
            if (mine) {
                ph.i = next + rank;
                const ms_medium m = J.media[J.per_photon_media ? ph.i : 0];
                ph.sig = (real)m.optical_radius;
                ph.g = (real)m.g;
                ph.phi = (real)m.albedo;
                ph.paper = m.first_event_at_origin != 0;
                ph.p = V3<Pol>{(real)0, (real)0, (real)0};
                ph.rep_p = ph.p;
                ph.rep_w = ph.p;
                ph.rep_k = 0;
                ph.pw = (real)1;
                ph.wsum = (real)0;
                ph.n = 0;
                ph.step = 0;
                const Stream s(J.seed, J.offset + ph.i);
                if (m.isotropic_start) {
                    real u[4];
                    if (ph.paper) {
                        Pol::uniforms(s, 0u, 1u, u);
                        ph.w = isotropic<Pol>(u[2], u[3]);
                    } else {
                        Pol::uniforms(s, 0u, 0u, u);
                        ph.w = isotropic<Pol>(u[1], u[2]);
                    }
                } else {
                    const real dx = (real)m.dir_in[0], dy = (real)m.dir_in[1], dz = (real)m.dir_in[2];
                    const real nn = Pol::sqrt(dx * dx + dy * dy + dz * dz);
                    ph.w = V3<Pol>{dx / nn, dy / nn, dz / nn};
                }
                active = true;
            }
            next += (need != 0u) ? (uint64_t)min((unsigned)__popc(need), avail) : 0ull;
            need = __ballot_sync(0xffffffffu, !active);
        }
        if (!__any_sync(0xffffffffu, active)) break;
        if (!active) continue;

        // ---- one scattering event and one free flight ----
        const Stream s(J.seed, J.offset + ph.i);
        real u[4], ures;
        Pol::uniforms(s, ph.step, 0u, u, &ures);
        int done = -1;
        if (ph.step > 0u || ph.paper) {
            if (ph.n >= J.max_events) {
                done = MS_TRUNCATED;
            } else {
                ph.n += 1u;
                if (J.reservoir) {
                    real wk;
                    if (J.reservoir == 1) {
                        wk = (real)1;
                    } else {
                        ph.pw = ph.pw * ph.phi;
                        wk = ph.pw;
                    }
                    ph.wsum = ph.wsum + wk;
                    if (ures * ph.wsum < wk) {
                        ph.rep_p = ph.p;
                        ph.rep_w = ph.w;
                        ph.rep_k = (int32_t)ph.n;
                    }
                }
                if (J.reservoir != 2 && u[3] >= ph.phi) {
                    done = MS_ABSORBED;
                } else {
                    ph.w = scatter<Pol>(ph.w, hg_cosine<Pol>(u[1], ph.g), u[2]);
                }
            }
        }
        V3<Pol> x{(real)0, (real)0, (real)0};
        if (done < 0) {
            const real l = Pol::div(-Pol::log((real)1 - u[0]), ph.sig);
            const real b = dot<Pol>(ph.p, ph.w);
            const real c = dot<Pol>(ph.p, ph.p) - (real)1;
            real disc = b * b - c;
            if (disc < (real)0) disc = (real)0;
            const real te = -b + Pol::sqrt(disc);
            if (l >= te) {
                x = V3<Pol>{ph.p.x + te * ph.w.x, ph.p.y + te * ph.w.y, ph.p.z + te * ph.w.z};
                x = unit<Pol>(x);
                done = MS_ESCAPED;
            } else {
                ph.p = V3<Pol>{ph.p.x + l * ph.w.x, ph.p.y + l * ph.w.y, ph.p.z + l * ph.w.z};
            }
        }
        ph.step += 1u;
        if (done < 0) continue;

        // ---- the photon is finished: histograms and records ----
        active = false;
        my_events += ph.n;
        atomicAdd(&s_hist_n[hist_n_bin(ph.n)], 1u);
        if (done == MS_ESCAPED) {
            ++my_escaped;
            const int bi = clampi((int)((x.z + (real)1) * (real)16), 0, 31);
            const real az = Pol::atan2(x.y, x.x);
            const int bj = clampi((int)((az + Pol::kPi) / Pol::kTwoPi * (real)64), 0, 63);
            atomicAdd(&s_hist_pos[bi * 64 + bj], 1u);
            const real mu_out = dot<Pol>(ph.w, x);
            atomicAdd(&s_hist_cos[clampi((int)(mu_out * (real)64), 0, 63)], 1u);
        } else if (done == MS_ABSORBED) {
            ++my_absorbed;
        } else {
            ++my_truncated;
        }
        const ms_walk_out& o = J.out;
        const uint64_t i = ph.i;
        if (o.n_events) o.n_events[i] = (int32_t)ph.n;
        if (o.status) o.status[i] = (uint8_t)done;
        if (o.exit_pos) {
            o.exit_pos[3 * i] = (float)x.x; o.exit_pos[3 * i + 1] = (float)x.y; o.exit_pos[3 * i + 2] = (float)x.z;
        }
        if (o.exit_dir) {
            const bool e = done == MS_ESCAPED;
            o.exit_dir[3 * i] = e ? (float)ph.w.x : 0.f;
            o.exit_dir[3 * i + 1] = e ? (float)ph.w.y : 0.f;
            o.exit_dir[3 * i + 2] = e ? (float)ph.w.z : 0.f;
        }
        if (o.rep_pos) {
            o.rep_pos[3 * i] = (float)ph.rep_p.x; o.rep_pos[3 * i + 1] = (float)ph.rep_p.y;
            o.rep_pos[3 * i + 2] = (float)ph.rep_p.z;
        }
        if (o.rep_dir) {
            o.rep_dir[3 * i] = (float)ph.rep_w.x; o.rep_dir[3 * i + 1] = (float)ph.rep_w.y;
            o.rep_dir[3 * i + 2] = (float)ph.rep_w.z;
        }
        if (o.rep_index) o.rep_index[i] = ph.rep_k;
    }

    // ---- block totals -> global accumulators ----
    for (int off = 16; off > 0; off >>= 1) {
        my_escaped += __shfl_xor_sync(0xffffffffu, my_escaped, off);
        my_absorbed += __shfl_xor_sync(0xffffffffu, my_absorbed, off);
        my_truncated += __shfl_xor_sync(0xffffffffu, my_truncated, off);
        my_events += __shfl_xor_sync(0xffffffffu, my_events, off);
    }
    if (lane == 0) {
        atomicAdd(&s_cnt[0], my_escaped);
        atomicAdd(&s_cnt[1], my_absorbed);
        atomicAdd(&s_cnt[2], my_truncated);
        atomicAdd(&s_cnt[3], my_events);
    }
    __syncthreads();
    const ms_walk_out& o = J.out;
    if (o.hist_pos)
        for (int k = threadIdx.x; k < 32 * 64; k += kThreads)
            if (s_hist_pos[k]) atomicAdd(&o.hist_pos[k], (unsigned long long)s_hist_pos[k]);
    if (threadIdx.x < 64) {
        if (o.hist_n && s_hist_n[threadIdx.x]) atomicAdd(&o.hist_n[threadIdx.x], (unsigned long long)s_hist_n[threadIdx.x]);
        if (o.hist_cos && s_hist_cos[threadIdx.x])
            atomicAdd(&o.hist_cos[threadIdx.x], (unsigned long long)s_hist_cos[threadIdx.x]);
    }
    if (o.counters && threadIdx.x < 4 && s_cnt[threadIdx.x]) atomicAdd(&o.counters[threadIdx.x], s_cnt[threadIdx.x]);
}

// Launches one persistent walk over J.n photons (one resident wave of blocks); the ticket must be zero.
template <class Pol>
cudaError_t launch(const Job& J, cudaStream_t stream)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel<Pol>, kThreads, 0);
    if (e != cudaSuccess) return e;
    int grid = num_sms() * (per_sm > 0 ? per_sm : 1);
    const uint64_t max_useful = (J.n + kThreads - 1) / kThreads;
    if ((uint64_t)grid > max_useful) grid = (int)(max_useful > 0 ? max_useful : 1);
    walk_kernel<Pol><<<grid, kThreads, 0, stream>>>(J);
    return cudaGetLastError();
}

}  // namespace walk
}  // namespace ms
