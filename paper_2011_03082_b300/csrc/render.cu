// ms_render / ms_render_batch: sphere-traced (learned) and brute-force rendering of a homogeneous translucent
// SDF object with next-event estimation toward a point light.
//
// Method (Sec. 3 and Fig. 2b; Sec. 4.1, Eq. 3-4; Sec. 4.3, Eq. 5): a camera path enters the object and
// alternates free flights (exponential, the homogeneous case of delta tracking) with, at each collision,
// either one sphere-tracing step — the largest sphere inside the boundary from the SDF, LengthGen /
// absorption / PathGen / EventGen at the rescaled optical radius sigma_t r, NEE at the representative event
// with weight Lambda^(N) — or, in thin regions and in brute-force mode, one scattering event with NEE weight
// phi, Russian roulette and HG scattering.
//
// Kernel design (persistent, one launch for any number of requests):
//  * each block owns 256 path slots, one per thread; slots are refilled from a global ticket of camera
//    samples with one warp-aggregated atomic per refill round;
//  * a block iteration is a wavefront of stages separated by barriers: (1) refill, (2) flight by the owning
//    thread (SDF sphere-tracing march inside, and outside on exit to find a re-entry), brute-force events
//    in place, (3) the sphere steps, compacted into a shared-memory queue with __ballot_sync / __popc and a
//    block prefix so the three decoder MLPs run on full warps, (4) next-event estimation (shadow march) by
//    the owning thread;
//  * the decoder weights of all three models sit in shared memory (broadcast float4 loads, decoder.cuh);
//  * a path's contributions accumulate in a register in double precision and are added to its pixel once,
//    when the path ends; per-request counters are shared-memory atomics flushed at block exit;
//  * every loop is bounded: segments per path, march steps per march, and the block loop ends when the
//    ticket is drained and no slot is live.
#include <cmath>

#include "decoder.cuh"
#include "ms_device.cuh"

namespace ms {
namespace render {

constexpr int kThreads = 256;
constexpr int kMaxReq = 64;
constexpr int kStats = MS_RENDER_STATS;
constexpr float kEps = 1e-4f;       // distance from the boundary treated as on it
constexpr int kMaxMarch = 1024;     // sphere-tracing steps per march; running out ends the path
constexpr float kNMax = 16777216.0f;

struct Req {
    float cam[3], at[3], tan_half, aspect;
    float light[3], I;
    float sigma, g, phi, log_phi, A, k, lip, rb2;
    float tau_min, tau_max;
    int32_t W, H, mode;
    uint32_t spp, max_segments;
    uint64_t seed, sample_offset, image_offset, samples_begin;
};

struct Batch {
    int n;
    uint64_t total;
    Req r[kMaxReq];
    const float* wL;     // decoder weights (packed float32) LengthGen, PathGen, EventGen; null in brute force
    const float* wP;
    const float* wE;
    double* image;
    unsigned long long* stats;   // [n][kStats]
    unsigned long long* ticket;
};

// decoder shapes: LengthGen (2 + 4 -> 1), PathGen (3 + 4 -> 3), EventGen (7 + 4 -> 6)
constexpr int kInL = 8, kPL = 1, kInP = 8, kPP = 3, kInE = 12, kPE = 6;
constexpr int kSmemL = dec::smem_floats(kInL, kPL), kSmemP = dec::smem_floats(kInP, kPP),
              kSmemE = dec::smem_floats(kInE, kPE);

struct V { float x, y, z; };
__device__ __forceinline__ V v3(float x, float y, float z) { return V{x, y, z}; }
__device__ __forceinline__ V operator+(V a, V b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V operator-(V a, V b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V operator*(V a, float s) { return v3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot(V a, V b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V cross(V a, V b) { return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ V unit(V a) { return a * rsqrtf(dot(a, a)); }

// per-thread SDF evaluation counters (distance, gradient), flushed into the request's stats
struct Evals { unsigned f, g; };

// ---- the displaced sphere f(p) = |p| - 1 - A sin(kx) sin(ky) sin(kz) (negative inside) ----
__device__ __forceinline__ float sdf(const Req& q, V p, Evals& ev)
{
    ++ev.f;
    return sqrtf(dot(p, p)) - 1.0f - q.A * __sinf(q.k * p.x) * __sinf(q.k * p.y) * __sinf(q.k * p.z);
}

__device__ __forceinline__ V sdf_grad(const Req& q, V p, Evals& ev)
{
    ++ev.g;
    float sx, cx, sy, cy, sz, cz;
    __sincosf(q.k * p.x, &sx, &cx);
    __sincosf(q.k * p.y, &sy, &cy);
    __sincosf(q.k * p.z, &sz, &cz);
    const float inv = rsqrtf(dot(p, p));
    const float ak = q.A * q.k;
    return v3(p.x * inv - ak * cx * sy * sz, p.y * inv - ak * sx * cy * sz, p.z * inv - ak * sx * sy * cz);
}

// 1: collision at *c = p + l w; 0: crossed the boundary outward at *c; 2: step cap
__device__ int march_inside(const Req& q, V p, V w, float l, V* c, Evals& ev)
{
    float t = 0.0f;
    for (int it = 0; it < kMaxMarch; ++it) {
        const V r = p + w * t;
        float d = -sdf(q, r, ev) / q.lip;
        if (d < kEps) {
            if (dot(sdf_grad(q, r, ev), w) > 0.0f) { *c = r; return 0; }
            d = kEps;
        }
        if (t + d >= l) { *c = p + w * l; return 1; }
        t += d;
    }
    return 2;
}

// 1: re-entered at *c; 0: left the bounding sphere; 2: step cap
__device__ int march_outside(const Req& q, V p, V w, V* c, Evals& ev)
{
    float t = 0.0f;
    for (int it = 0; it < kMaxMarch; ++it) {
        const V r = p + w * t;
        if (dot(r, r) > q.rb2 && dot(r, w) >= 0.0f) return 0;
        float d = sdf(q, r, ev) / q.lip;
        if (d < kEps) {
            if (dot(sdf_grad(q, r, ev), w) < 0.0f) { *c = r; return 1; }
            d = kEps;
        }
        t += d;
    }
    return 2;
}

// length of X -> light inside the medium (Sec. 4.3 d_t); negative when the step cap runs out
__device__ float inside_length(const Req& q, V X, V xl, Evals& ev)
{
    const V dl = xl - X;
    const float D = sqrtf(dot(dl, dl));
    const V w = dl * (1.0f / D);
    float t = 0.0f, din = 0.0f;
    bool inside = true;
    for (int it = 0; it < kMaxMarch; ++it) {
        if (t >= D) return din;
        const V r = X + w * t;
        const float f = sdf(q, r, ev);
        if (inside) {
            float d = -f / q.lip;
            if (d < kEps) {
                if (dot(sdf_grad(q, r, ev), w) > 0.0f) { inside = false; continue; }
                d = kEps;
            }
            const float step = fminf(d, D - t);
            din += step;
            t += step;
        } else {
            if (dot(r, r) > q.rb2 && dot(r, w) >= 0.0f) return din;
            float d = f / q.lip;
            if (d < kEps) {
                if (dot(sdf_grad(q, r, ev), w) < 0.0f) { inside = true; continue; }
                d = kEps;
            }
            t += fminf(d, D - t);
        }
    }
    return -1.0f;
}

__device__ __forceinline__ float hg_pdf(float cosang, float g)
{
    const float den = 1.0f + g * g - 2.0f * g * cosang;
    return (1.0f - g * g) * 0.0795774715459476679f * rsqrtf(den) / den;
}

__device__ __forceinline__ float hg_cosine(float u, float g)
{
    if (fabsf(g) < 1e-4f) return 2.0f * u - 1.0f;
    const float t = __fdividef(1.0f - g * g, 1.0f - g + 2.0f * g * u);
    return fminf(1.0f, fmaxf(-1.0f, __fdividef(1.0f + g * g - t * t, 2.0f * g)));
}

__device__ __forceinline__ void onb(V w, V* t1, V* t2)
{
    const float sign = w.z >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (sign + w.z);
    const float b = w.x * w.y * a;
    *t1 = v3(1.0f + sign * w.x * w.x * a, sign * b, -sign * w.x);
    *t2 = v3(b, sign + w.y * w.y * a, -w.y);
}

__device__ __forceinline__ V scatter_dir(V w, float mu, float u)
{
    V t1, t2;
    onb(w, &t1, &t2);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
    float sp, cp;
    sincos_turns_fast(u, &sp, &cp);
    return unit(t1 * (st * cp) + t2 * (st * sp) + w * mu);
}

// Camera ray of sample (pixel, jitter) of request q.
__device__ __forceinline__ void camera_ray(const Req& q, int px, int py, float jx, float jy, V* o, V* d)
{
    const V cp = v3(q.cam[0], q.cam[1], q.cam[2]);
    const V fw = unit(v3(q.at[0], q.at[1], q.at[2]) - cp);
    const V rt = unit(cross(fw, v3(0.0f, 1.0f, 0.0f)));
    const V up = cross(rt, fw);
    const float sx = (2.0f * ((float)px + jx) / (float)q.W - 1.0f) * q.tan_half * q.aspect;
    const float sy = (1.0f - 2.0f * ((float)py + jy) / (float)q.H) * q.tan_half;
    *o = cp;
    *d = unit(fw + rt * sx + up * sy);
}

// per-slot data exchanged with the sphere stage
struct SphereJob {
    float c[3], w[3], r, tau;
    uint32_t id_lo, id_hi, seg, req;
};
struct SphereOut {
    float X[3], W[3], lam, p[3], w[3];
    int absorbed;
};

__device__ __forceinline__ int find_req(const Batch& B, uint64_t t)
{
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.r[mid].samples_begin <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads, 1) render_kernel(const __grid_constant__ Batch B)
{
    __shared__ __align__(16) float sw[kSmemL + kSmemP + kSmemE];
    __shared__ SphereJob s_job[kThreads];
    __shared__ SphereOut s_out[kThreads];
    __shared__ int s_queue[kThreads];
    __shared__ int s_warp_count[kThreads / 32];
    __shared__ int s_nq;
    __shared__ unsigned long long s_stats[kMaxReq * kStats];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool learned = B.wL != nullptr;
    float* wl = sw;
    float* wpth = sw + kSmemL;
    float* wev = sw + kSmemL + kSmemP;
    if (learned) {
        dec::stage_weights(wl, B.wL, 2 + 4, kInL, kPL);
        dec::stage_weights(wpth, B.wP, 3 + 4, kInP, kPP);
        dec::stage_weights(wev, B.wE, 7 + 4, kInE, kPE);
    }
    for (int k = tid; k < kMaxReq * kStats; k += kThreads) s_stats[k] = 0ull;
    __syncthreads();

    // slot state (owned by this thread)
    bool live = false;
    int req = 0;
    uint32_t id_lo = 0, id_hi = 0, seg = 0;
    V p = v3(0, 0, 0), w = v3(0, 0, 1);
    double acc = 0.0;
    bool drained = false;   // warp-uniform
    Evals ev{0u, 0u};

    auto stat = [&](int r, int k, unsigned long long v) { atomicAdd(&s_stats[r * kStats + k], v); };
    auto flush_evals = [&](int r) {
        if (ev.f) stat(r, 8, ev.f);
        if (ev.g) stat(r, 9, ev.g);
        ev.f = ev.g = 0u;
    };
    auto finish = [&]() {
        flush_evals(req);
        if (acc != 0.0) {
            const Req& q = B.r[req];
            atomicAdd(&B.image[q.image_offset + id_hi], acc);
        }
        acc = 0.0;
        live = false;
    };

    for (;;) {
        // ---------------- (1) refill free slots with new camera samples ----------------
        bool need = !live;
        for (;;) {
            const unsigned m = __ballot_sync(0xffffffffu, need && !drained);
            if (m == 0u) break;
            unsigned long long base = 0;
            const int leader = __ffs(m) - 1;
            if (lane == leader) base = atomicAdd(B.ticket, (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (base + __popc(m) >= B.total) drained = true;
            if (need && ((m >> lane) & 1u)) {
                const uint64_t t = base + __popc(m & ((1u << lane) - 1u));
                if (t < B.total) {
                    const int r = find_req(B, t);
                    const Req& q = B.r[r];
                    const uint64_t local = t - q.samples_begin;
                    const uint32_t pixel = (uint32_t)(local / q.spp);
                    const uint32_t sample = (uint32_t)(q.sample_offset + local % q.spp);
                    const Stream st(q.seed, ((uint64_t)pixel << 32) | sample);
                    const Words j = st.at(0u, 8u);
                    V o, d;
                    camera_ray(q, (int)(pixel % (uint32_t)q.W), (int)(pixel / (uint32_t)q.W), u24(j.w0), u24(j.w1),
                               &o, &d);
                    stat(r, 0, 1ull);
                    V hit;
                    const int h = march_outside(q, o, d, &hit, ev);
                    if (h == 1) {
                        stat(r, 1, 1ull);
                        live = true;
                        need = false;
                        req = r;
                        id_lo = sample;
                        id_hi = pixel;
                        seg = 0;
                        p = hit;
                        w = d;
                        acc = 0.0;
                    } else {
                        if (h == 2) stat(r, 6, 1ull);
                        flush_evals(r);
                    }
                } else {
                    need = false;
                }
            }
        }
        if (!__syncthreads_or(live)) break;

        // ---------------- (2) flight; brute-force events in place ----------------
        const Req& q = B.r[req];
        bool sphere = false, nee_req = false, end_after_nee = false;
        V nX = v3(0, 0, 0), nW = v3(0, 0, 1);
        float nwt = 0.0f;
        if (live) {
            if (seg >= q.max_segments) {
                stat(req, 6, 1ull);
                finish();
            } else {
                stat(req, 2, 1ull);
                const Stream st(q.seed, ((uint64_t)id_hi << 32) | id_lo);
                const Words u = st.at(seg, 0u);
                const float l = -__logf(1.0f - u24(u.w0)) / q.sigma;
                V c;
                const int ev_kind = march_inside(q, p, w, l, &c, ev);
                if (ev_kind == 2) {
                    stat(req, 6, 1ull);
                    finish();
                } else if (ev_kind == 0) {
                    V re;
                    const int back = march_outside(q, c, w, &re, ev);
                    if (back == 1) {
                        p = re;
                        ++seg;
                    } else {
                        if (back == 2) stat(req, 6, 1ull);
                        finish();
                    }
                } else {
                    bool done_event = false;
                    if (q.mode == MS_SPHERE && learned) {
                        const float d = -sdf(q, c, ev) / q.lip;
                        const float r = fminf(d, q.tau_max / q.sigma);
                        const float tau = q.sigma * r;
                        if (tau >= q.tau_min) {
                            sphere = true;
                            done_event = true;
                            SphereJob& jb = s_job[tid];
                            jb.c[0] = c.x; jb.c[1] = c.y; jb.c[2] = c.z;
                            jb.w[0] = w.x; jb.w[1] = w.y; jb.w[2] = w.z;
                            jb.r = r; jb.tau = tau;
                            jb.id_lo = id_lo; jb.id_hi = id_hi; jb.seg = seg; jb.req = (uint32_t)req;
                        }
                    }
                    if (!done_event) {
                        stat(req, 4, 1ull);
                        nee_req = true;
                        nX = c;
                        nW = w;
                        nwt = q.phi;
                        if (u24(u.w3) >= q.phi) {
                            stat(req, 5, 1ull);
                            end_after_nee = true;
                        } else {
                            w = scatter_dir(w, hg_cosine(u24(u.w1), q.g), u24(u.w2));
                            p = c;
                            ++seg;
                        }
                    }
                }
            }
        }

        // ---------------- (3) sphere steps: ballot-compacted queue, decoders on full warps ----------------
        const unsigned mask = __ballot_sync(0xffffffffu, sphere);
        if (lane == 0) s_warp_count[warp] = __popc(mask);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < kThreads / 32; ++k) {
            const int c = s_warp_count[k];
            before += k < warp ? c : 0;
            total += c;
        }
        if (sphere) s_queue[before + __popc(mask & ((1u << lane) - 1u))] = tid;
        __syncthreads();
        if (tid < total) {
            const int slot = s_queue[tid];
            const SphereJob jb = s_job[slot];
            const Req& qq = B.r[jb.req];
            stat(jb.req, 3, 1ull);
            const Stream st(qq.seed, ((uint64_t)jb.id_hi << 32) | jb.id_lo);
            const Words a4 = st.at(jb.seg, 1u);
            float n[24];
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                const float4 v = dec::normals4(st, jb.seg, 2u + t);
                n[4 * t] = v.x; n[4 * t + 1] = v.y; n[4 * t + 2] = v.z; n[4 * t + 3] = v.w;
            }
            const float ltau = __logf(jb.tau);
            // LengthGen: N (phi = 1 physics, Eq. 3)
            float xin8[8] = {ltau, qq.g, n[0], n[1], n[2], n[3], 0.0f, 0.0f};
            float y4[4];
            dec::mlp<kInL, kPL>(wl, xin8, y4);
            const float yN = y4[0] + __expf(0.5f * y4[1]) * n[4];
            float N = floorf(__expf(yN) + 0.5f);
            N = fminf(fmaxf(N, 1.0f), kNMax);
            const float lnN = __logf(N);
            // PathGen: (cos theta, alpha, beta)
            float xp8[8] = {ltau, qq.g, lnN, n[5], n[6], n[7], n[8], 0.0f};
            float y8[8];
            dec::mlp<kInP, kPP>(wpth, xp8, y8);
            const float ct = fminf(1.0f, fmaxf(-1.0f, y8[0] + __expf(0.5f * y8[3]) * n[9]));
            float al = y8[1] + __expf(0.5f * y8[4]) * n[10];
            float be = y8[2] + __expf(0.5f * y8[5]) * n[11];
            float ab2 = al * al + be * be;
            if (ab2 > 1.0f) {
                const float s = rsqrtf(ab2);
                al *= s; be *= s; ab2 = 1.0f;
            }
            // EventGen: representative event (X~, W~)
            float xe12[12] = {ltau, qq.g, qq.phi, ct, al, be, lnN, n[12], n[13], n[14], n[15], 0.0f};
            float y12[12];
            dec::mlp<kInE, kPE>(wev, xe12, y12);
            float e[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) e[k] = y12[k] + __expf(0.5f * y12[6 + k]) * n[16 + k];
            const float phiN = __expf(N * qq.log_phi);
            const float lam = qq.phi < 1.0f ? qq.phi * (1.0f - phiN) / (1.0f - qq.phi) : N;
            // Eq. 4 and Sec. 4.1: CVAE frame -> world via R^CVAE R_psi, scaled by r
            const V wi = v3(jb.w[0], jb.w[1], jb.w[2]);
            V t1, t2;
            onb(wi, &t1, &t2);
            float sn, cs;
            sincos_turns_fast(u24(a4.w1), &sn, &cs);
            const float stt = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
            const float nn = sqrtf(fmaxf(0.0f, 1.0f - ab2));
            V vs[4] = {v3(stt, 0.0f, ct), v3(be * ct + nn * stt, al, -be * stt + nn * ct), v3(e[0], e[1], e[2]),
                       v3(e[3], e[4], e[5])};
            const float xn2 = dot(vs[2], vs[2]);
            if (xn2 > 1.0f) vs[2] = vs[2] * rsqrtf(xn2);
            const float wn2 = dot(vs[3], vs[3]);
            vs[3] = wn2 > 1e-24f ? vs[3] * rsqrtf(wn2) : v3(0.0f, 0.0f, 1.0f);
            V vw[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const V v1 = v3(cs * vs[k].x - sn * vs[k].y, sn * vs[k].x + cs * vs[k].y, vs[k].z);
                vw[k] = t1 * v1.x + t2 * v1.y + wi * v1.z;
            }
            const V c = v3(jb.c[0], jb.c[1], jb.c[2]);
            const V xexit = c + vw[0] * jb.r;
            const V wout = unit(vw[1]);
            const V X = c + vw[2] * jb.r;
            const V Wd = unit(vw[3]);
            SphereOut& so = s_out[slot];
            so.X[0] = X.x; so.X[1] = X.y; so.X[2] = X.z;
            so.W[0] = Wd.x; so.W[1] = Wd.y; so.W[2] = Wd.z;
            so.lam = lam;
            so.p[0] = xexit.x; so.p[1] = xexit.y; so.p[2] = xexit.z;
            so.w[0] = wout.x; so.w[1] = wout.y; so.w[2] = wout.z;
            so.absorbed = u24(a4.w0) >= phiN;
        }
        __syncthreads();
        if (sphere) {
            const SphereOut so = s_out[tid];
            nee_req = true;
            nX = v3(so.X[0], so.X[1], so.X[2]);
            nW = v3(so.W[0], so.W[1], so.W[2]);
            nwt = so.lam;
            if (so.absorbed) {
                stat(req, 5, 1ull);
                end_after_nee = true;
            } else {
                p = v3(so.p[0], so.p[1], so.p[2]);
                w = v3(so.w[0], so.w[1], so.w[2]);
                ++seg;
            }
        }

        // ---------------- (4) next-event estimation toward the point light (Eq. 5 term) ----------------
        if (nee_req) {
            stat(req, 7, 1ull);
            const V xl = v3(q.light[0], q.light[1], q.light[2]);
            const V dl = xl - nX;
            const float d2 = dot(dl, dl);
            const V wl2 = dl * rsqrtf(d2);
            const float din = inside_length(q, nX, xl, ev);
            if (din < 0.0f) {
                stat(req, 6, 1ull);
            } else {
                const float rho = hg_pdf(dot(nW, wl2), q.g);
                acc += (double)(nwt * rho * __expf(-q.sigma * din) * q.I / d2);
            }
            if (end_after_nee) finish();
        }
        __syncthreads();
    }

    // ---------------- per-request counters -> global ----------------
    for (int k = tid; k < B.n * kStats; k += kThreads)
        if (s_stats[k]) atomicAdd(&B.stats[k], s_stats[k]);
}

}  // namespace render
}  // namespace ms

using namespace ms::render;

static ms_status fill_batch(const ms_render_params* reqs, int n, Batch* b, const char* fn)
{
    if (n < 1 || n > kMaxReq) return ms::set_error(MS_ERR_INVALID_ARG, "%s: 1..%d requests per call", fn, kMaxReq);
    uint64_t samples = 0, pixels = 0;
    b->n = n;
    for (int i = 0; i < n; ++i) {
        const ms_render_params& p = reqs[i];
        if (p.width < 1 || p.height < 1 || p.spp < 1)
            return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: width, height and spp must be >= 1", fn, i);
        if (!(p.sigma_t > 0.0f) || !(p.g > -1.0f && p.g < 1.0f) || !(p.albedo >= 0.0f && p.albedo <= 1.0f))
            return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: need sigma_t > 0, |g| < 1, albedo in [0,1]",
                                 fn, i);
        if (!(p.disp_amp >= 0.0f) || !(p.disp_freq >= 0.0f) || !(p.fov_y_deg > 0.0f && p.fov_y_deg < 180.0f))
            return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: bad displacement or field of view", fn, i);
        if (p.mode != MS_BRUTE && p.mode != MS_SPHERE)
            return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: mode must be MS_BRUTE or MS_SPHERE", fn, i);
        if (p.max_segments < 1) return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: max_segments >= 1", fn, i);
        if ((uint64_t)p.width * p.height >= (1ull << 32) || p.sample_offset + p.spp > (1ull << 32))
            return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: pixel or sample index exceeds 32 bits", fn, i);
        Req& q = b->r[i];
        for (int k = 0; k < 3; ++k) {
            q.cam[k] = p.cam_pos[k];
            q.at[k] = p.cam_at[k];
            q.light[k] = p.light_pos[k];
        }
        q.tan_half = (float)std::tan(0.5 * (double)p.fov_y_deg * 3.14159265358979323846 / 180.0);
        q.aspect = (float)p.width / (float)p.height;
        q.I = p.light_I;
        q.sigma = p.sigma_t;
        q.g = p.g;
        q.phi = p.albedo;
        q.log_phi = p.albedo > 0.0f ? std::log(p.albedo) : -INFINITY;
        q.A = p.disp_amp;
        q.k = p.disp_freq;
        q.lip = 1.0f + p.disp_amp * p.disp_freq;
        const float rb = 1.0f + p.disp_amp + 1e-3f;
        q.rb2 = rb * rb;
        q.tau_min = p.min_optical_radius;
        q.tau_max = p.max_optical_radius;
        q.W = p.width;
        q.H = p.height;
        q.mode = p.mode;
        q.spp = p.spp;
        q.max_segments = p.max_segments;
        q.seed = p.seed;
        q.sample_offset = p.sample_offset;
        q.image_offset = pixels;
        q.samples_begin = samples;
        pixels += (uint64_t)p.width * p.height;
        samples += (uint64_t)p.width * p.height * p.spp;
    }
    b->total = samples;
    return MS_OK;
}

extern "C" size_t ms_render_workspace_size(const ms_render_params* reqs, int n_requests)
{
    (void)reqs;
    (void)n_requests;
    return 256;
}

static ms_status render_launch(const ms_render_params* reqs, int n, const ms_cvae_set* models, double* images,
                               unsigned long long* stats, void* workspace, size_t workspace_bytes, void* stream,
                               const char* fn)
{
    MS_CHECK_ARG(reqs != nullptr && images != nullptr && stats != nullptr, "%s: null argument", fn);
    MS_CHECK_ARG(workspace != nullptr && workspace_bytes >= 256 && ((uintptr_t)workspace & 255u) == 0,
                 "%s: a 256-byte aligned workspace of at least 256 bytes is required", fn);
    Batch b;
    ms_status st = fill_batch(reqs, n, &b, fn);
    if (st != MS_OK) return st;
    bool any_sphere = false;
    for (int i = 0; i < n; ++i) any_sphere |= reqs[i].mode == MS_SPHERE;
    b.wL = b.wP = b.wE = nullptr;
    if (any_sphere) {
        MS_CHECK_ARG(models != nullptr, "%s: MS_SPHERE needs the three decoders", fn);
        const ms_decoder* d[3] = {&models->length, &models->path, &models->event};
        const int pin[3] = {2, 3, 7}, pout[3] = {1, 3, 6};
        for (int k = 0; k < 3; ++k) {
            MS_CHECK_ARG(d[k]->weights != nullptr && d[k]->p_in == pin[k] && d[k]->p_out == pout[k] &&
                             d[k]->latent == 4 && d[k]->width == 16,
                         "%s: decoder %d must have p_in %d, latent 4, width 16, p_out %d", fn, k, pin[k], pout[k]);
            MS_CHECK_ARG(d[k]->precision == MS_FP32, "%s: the renderer evaluates FP32 decoders", fn);
        }
        b.wL = models->length.weights;
        b.wP = models->path.weights;
        b.wE = models->event.weights;
    }
    b.image = images;
    b.stats = stats;
    b.ticket = static_cast<unsigned long long*>(workspace);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MS_CUDA(cudaMemsetAsync(workspace, 0, sizeof(unsigned long long), s));
    int per_sm = 0;
    MS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_kernel, kThreads, 0));
    uint64_t grid = (uint64_t)ms::num_sms() * (per_sm > 0 ? per_sm : 1);
    const uint64_t need = (b.total + kThreads - 1) / kThreads;
    if (grid > need) grid = need;
    render_kernel<<<(unsigned)grid, kThreads, 0, s>>>(b);
    MS_CUDA(cudaGetLastError());
    return MS_OK;
}

extern "C" ms_status ms_render(const ms_render_params* p, const ms_cvae_set* models, double* image,
                               unsigned long long* stats, void* workspace, size_t workspace_bytes, void* stream)
{
    return render_launch(p, 1, models, image, stats, workspace, workspace_bytes, stream, "ms_render");
}

extern "C" ms_status ms_render_batch(const ms_render_params* reqs, int n, const ms_cvae_set* models, double* images,
                                     unsigned long long* stats, void* workspace, size_t workspace_bytes,
                                     void* stream)
{
    return render_launch(reqs, n, models, images, stats, workspace, workspace_bytes, stream, "ms_render_batch");
}
