// ms_render / ms_render_batch: sphere-traced (learned) and brute-force rendering of a homogeneous translucent
// SDF object with next-event estimation toward a point light.
//
// Method (Sec. 3 and Fig. 2b; Sec. 4.1, Eq. 3-4; Sec. 4.3, Eq. 5): a camera path enters the object and
// alternates free flights (exponential: the homogeneous case of delta tracking) with, at each collision,
// either one sphere-tracing step — the largest sphere inside the boundary from the SDF, LengthGen /
// absorption / PathGen / EventGen at the rescaled optical radius sigma_t r, NEE at the representative event
// with weight Lambda^(N) — or, in thin regions and in brute-force mode, one scattering event with NEE weight
// phi, Russian roulette and HG scattering.
//
// Kernel design (persistent; one launch for any number of requests; warps fully independent):
//  * every lane owns one path and runs a small state machine — camera march, free-flight march, re-entry
//    march, shadow march, decode — advancing one signed-distance step per loop iteration, so a warp stays
//    converged on the same short loop body however long the individual marches are; a lane whose path ends
//    takes the next camera sample at once (warp-aggregated ticket);
//  * a lane that reaches a sphere step parks in the decode state; the warp runs the three decoder MLPs only
//    when at least kDecodeBatch of its lanes are parked (or nothing else is marching), on one 16-row
//    tensor-core tile of up to 16 parked lanes (weights in shared memory in fragment order, decoder_mma.cuh),
//    while the other lanes keep marching, with no block or grid barrier in the loop;
//  * a path's NEE sum is kept in a register and added to its pixel (double) once; counters are per-lane
//    registers that run over the lane's paths of one request and are flushed to shared, then global, memory
//    when the lane changes request or finishes;
//  * everything is bounded: segments per path, steps per march, and the loop ends when the ticket is drained
//    and no lane holds a path.
//
// This header holds the kernel template; render.cu (host side, FP32 decoders and brute force), render_f16.cu and
// render_bf16.cu instantiate it, one translation unit per decoder precision so that they compile in parallel.
#pragma once

#include <cmath>

#include "decoder_mma.cuh"
#include "ms_device.cuh"

namespace ms {
namespace render {

constexpr int kThreads = 256;
constexpr int kMaxReq = 64;
constexpr int kStats = MS_RENDER_STATS;
constexpr float kEps = 1e-4f;       // distance from the boundary treated as on it
constexpr int kMaxMarch = 1024;     // steps per march; running out ends the path (or drops the estimate)
constexpr float kNMax = 16777216.0f;
constexpr float kTauCut = 30.0f;    // a shadow ray stops once its optical depth inside the medium exceeds this

struct Req {
    float cam[3], at[3], tan_half, aspect, two_over_w, two_over_h;
    float light[3], I;
    float sigma, inv_sigma, din_cut, g, phi, log_phi, A, k, lip, inv_lip, rb2;
    float tau_min, tau_max;
    const float* grid;               // voxel grid of conservative distances, or null
    int32_t grid_n;
    float grid_b, grid_inv_h;
    int32_t W, H, mode, exact_n1, exact_centre;
    uint32_t spp, max_segments;
    uint64_t seed, sample_offset, image_offset, samples_begin;
};

struct Batch {
    int n;
    uint64_t total;
    Req r[kMaxReq];
    const float* wL;                 // decoder weights LengthGen, PathGen, EventGen (null: brute force only)
    const float* wP;
    const float* wE;
    double* image;
    unsigned long long* stats;       // [n][kStats]
    unsigned long long* ticket;      // workspace: sample ticket, start time, finished paths per request
    unsigned long long* t_start;
    unsigned long long* done;        // [kMaxReq]
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// decoder shapes, the final settings of Table 1: LengthGen (2 + L 2 -> 1, width 8), PathGen (3 + L 5 -> 3,
// width 16), EventGen (7 + L 5 -> 6, width 16); tensor-core fragment layouts in shared memory
// (decoder_mma.cuh).  A sphere step's 22 normals n[] (tags 2..7) are split as z then eps per model.
constexpr int kLatL = 2, kLatP = 5, kLatE = 5;
constexpr int kZL = 0, kEL = kZL + kLatL, kZP = kEL + 1, kEP = kZP + kLatP, kZE = kEP + 3, kEE = kZE + kLatE;
static_assert(kEE + 6 <= 24, "a sphere step draws 24 normals");
constexpr int kBytesL = mmadec::smem_bytes(1, 1), kBytesP = mmadec::smem_bytes(3, 2),
              kBytesE = mmadec::smem_bytes(6, 2);

struct V { float x, y, z; };
__device__ __forceinline__ V v3(float x, float y, float z) { return V{x, y, z}; }
__device__ __forceinline__ V operator+(V a, V b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V operator-(V a, V b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V operator*(V a, float s) { return v3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot(V a, V b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V cross(V a, V b) { return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ V unit(V a) { return a * rsqrtf(dot(a, a)); }

// The constants of the march held in registers for the lane's current request.
struct Geo {
    float A, k, inv_lip, rb2, din_cut;
};

// ---- the displaced sphere f(p) = |p| - R(p), R(p) = 1 + A sin(kx) sin(ky) sin(kz) (negative inside) ----
__device__ __forceinline__ float sdf_parts(const Geo& q, V p, float* rp, float* R0)
{
    const float d2 = dot(p, p);
    *rp = d2 > 0.0f ? d2 * rsqrtf(d2) : 0.0f;
    *R0 = fmaf(q.A, __sinf(q.k * p.x) * __sinf(q.k * p.y) * __sinf(q.k * p.z), 1.0f);
    return *rp - *R0;
}

__device__ __forceinline__ float sdf(const Geo& q, V p)
{
    float rp, R0;
    return sdf_parts(q, p, &rp, &R0);
}

// Step along w from p that cannot cross the surface: the displacement A sin sin sin is (A k)-Lipschitz and
// the radial term |p + s w| is exact along the ray, so with lam = A k and R0 = R(p) the surface is not
// reached before |p + s w| = R0 + lam s (outside) or R0 - lam s (inside).  Squared, that is
// a s^2 + 2 B s + c = 0 with a = 1 - lam^2, B = p.w -/+ R0 lam, c = |p|^2 - R0^2 = f (|p| + R0); the step is
// its first positive root, in the form without cancellation for the sign of B.  Outside, no positive root
// means the surface cannot be reached along the ray at all (*escape).
__device__ __forceinline__ float safe_step(const Geo& q, V p, V w, float rp, float R0, float f, bool in_medium,
                                           bool* escape)
{
    const float lam = q.A * q.k;
    const float a = fmaf(-lam, lam, 1.0f);
    const float c = f * (rp + R0);
    const float B = dot(p, w) + (in_medium ? R0 * lam : -R0 * lam);
    const float disc = fmaf(B, B, -a * c);
    const float sq = disc > 0.0f ? disc * rsqrtf(disc) : 0.0f;
    const bool pos = B >= 0.0f;
    // inside: B >= 0 ? -c / (B + sq) : (sq - B) / a;   outside: B < 0 ? c / (sq - B) : (B + sq) / -a
    const float num = in_medium ? (pos ? -c : sq - B) : (pos ? B + sq : c);
    const float den = in_medium ? (pos ? B + sq : a) : (pos ? -a : sq - B);
    *escape = !in_medium && (disc < 0.0f || (pos && a >= 0.0f));
    return __fdividef(num, den);
}

// The curvature step: with hs >= 0 the marched side's distance function (-f inside, f outside) and h1 its rate
// along the ray, the second directional derivative bound H = A k^2 (sin sin sin along a line is a sum of four
// sinusoids of angular frequencies k (+-w1 +-w2 +-w3), whose squares sum to 4 k^2) + 2 / |p| (inside only, the
// curvature of |p| while the step stays below |p| / 2) gives hs(s) >= hs + h1 s - H s^2 / 2 > 0 up to its
// first positive root, written without cancellation for the sign of h1.  Capped at |p| / 2 inside and 4
// outside (beyond the bounding sphere).  Toward the surface it closes in quadratically; away from it, it
// leaves the boundary band in one step.
__device__ __forceinline__ float curve_step(const Geo& q, float ir, float rp, float h0, float h1, bool in_medium)
{
    const float H = q.A * q.k * q.k + (in_medium ? 2.0f * ir : 0.0f);     // ir = 1 / |p|
    const float cap = in_medium ? 0.5f * rp : 4.0f;
    const float x = fmaf(h1, h1, 2.0f * H * h0);
    const float sq = x > 0.0f ? x * rsqrtf(x) : 0.0f;
    const bool toward = h1 < 0.0f;
    const float num = toward ? 2.0f * h0 : h1 + sq;
    const float den = toward ? sq - h1 : H;
    return (toward || H > 0.0f) ? fminf(__fdividef(num, den), cap) : cap;
}

// f at p with its parts (|p|, 1 / |p| and R(p)) and its derivative along the unit direction w.
__device__ __forceinline__ float sdf_parts_grad(const Geo& q, V p, V w, float* rp, float* irp, float* R0, float* gd)
{
    const float d2 = dot(p, p);
    const float ir = d2 > 0.0f ? rsqrtf(d2) : 0.0f;
    *irp = ir;
    float sx, cx, sy, cy, sz, cz;
    __sincosf(q.k * p.x, &sx, &cx);
    __sincosf(q.k * p.y, &sy, &cy);
    __sincosf(q.k * p.z, &sz, &cz);
    *rp = d2 * ir;
    *R0 = fmaf(q.A, sx * sy * sz, 1.0f);
    const float ds = fmaf(cx * sy * sz, w.x, fmaf(sx * cy * sz, w.y, sx * sy * cz * w.z));
    *gd = fmaf(-q.A * q.k, ds, dot(p, w) * ir);
    return *rp - *R0;
}

__device__ __forceinline__ float hg_pdf(float cosang, float g)
{
    const float den = 1.0f + g * g - 2.0f * g * cosang;
    return (1.0f - g * g) * 0.0795774715459476679f * __fdividef(rsqrtf(den), den);
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
    const float a = __fdividef(-1.0f, sign + w.z);      // |sign + w.z| in [1, 2]
    const float b = w.x * w.y * a;
    *t1 = v3(1.0f + sign * w.x * w.x * a, sign * b, -sign * w.x);
    *t2 = v3(b, sign + w.y * w.y * a, -w.y);
}

__device__ __forceinline__ V scatter_dir(V w, float mu, float u)
{
    V t1, t2;
    onb(w, &t1, &t2);
    const float st = sqrt_approx(fmaxf(0.0f, 1.0f - mu * mu));
    float sp, cp;
    sincos_turns_fast(u, &sp, &cp);
    return unit(t1 * (st * cp) + t2 * (st * sp) + w * mu);
}

__device__ __forceinline__ void camera_ray(const Req& q, int px, int py, float jx, float jy, V* o, V* d)
{
    const V cp = v3(q.cam[0], q.cam[1], q.cam[2]);
    const V fw = unit(v3(q.at[0], q.at[1], q.at[2]) - cp);
    const V rt = unit(cross(fw, v3(0.0f, 1.0f, 0.0f)));
    const V up = cross(rt, fw);
    const float sx = (((float)px + jx) * q.two_over_w - 1.0f) * q.tan_half * q.aspect;
    const float sy = (1.0f - ((float)py + jy) * q.two_over_h) * q.tan_half;
    *o = cp;
    *d = unit(fw + rt * sx + up * sy);
}

__device__ __forceinline__ int find_req(const Batch& B, uint64_t t)
{
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.r[mid].samples_begin <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kUsedStats = 10;
constexpr int kDraws = 29 * 16;      // a decoder round's draws: value v of row r at [v * 16 + r]
constexpr int kDrawKeys = 0;         // staging-tile offset of the draw keys (5 words per row) in a decoder round
static_assert(kDrawKeys + 5 * 16 <= mmadec::kStageFloats, "decoder-round draw keys exceed the staging tile");

// Scheduling constants of a kernel variant (see ms_render_autotune): kDecodeBatch parked lanes trigger a
// decoder round, kTransBatch pending (or idle) lanes a transition (or refill) round, and between two
// scheduling decisions each marching lane advances kSteps signed-distance steps.

enum State : int { kIdle = 0, kCamera, kFlight, kReentry, kShadow, kDecode, kPending };
enum Event : int { kEvHit = 0, kEvReenter, kEvEscape, kEvCap, kEvExit, kEvCollide, kEvShadowDone };

// kDec: the decoders' arithmetic, or 0 when the launch holds no sphere-tracing request: the brute-force
// instantiation carries no decoder code, which leaves its march and transitions free of register spills.
//   kDecFP32: weights and activations split into FP16 head + tail, three products per tile (about 22
//             significant bits: single-precision results);
//   kDecFP16 / kDecBF16: weights rounded once to FP16 / BF16, activations carried as head + tail (two products
//             per tile), FP32 accumulation: the error is that of the rounded weights.
enum : int { kDecNone = 0, kDecFP32 = 1, kDecFP16 = 2, kDecBF16 = 3 };

//
// kTimers: an instrumented instantiation for the time breakdown (ms_render_params.phase_timers): each warp
// accumulates clock64 cycles by round kind, added to the first request's stats[12..15] (march, decoder,
// transition, refill rounds, summed over warps), and march steps of shadow rays are counted in each request's
// stats[11].  The timed kernels are the kTimers = false instantiations, which carry none of this.
template <int kDecodeBatch, int kTransBatch, int kSteps, int kMinBlocks, int kDec, bool kTimers = false>
__global__ void __launch_bounds__(kThreads, kMinBlocks) render_kernel(const __grid_constant__ Batch B)
{
    constexpr bool kLearned = kDec != kDecNone;
    constexpr bool kHalfBF16 = kDec == kDecBF16;              // the half type of the tensor-core products
    constexpr int kSplit = kDec == kDecFP32 ? 3 : 2;
    constexpr int kRefillBatch = kTransBatch;
    __shared__ __align__(16) unsigned char sw[kBytesL + kBytesP + kBytesE];
    __shared__ float s_stage[kThreads / 32][mmadec::kStageFloats];
    __shared__ float s_draws[kLearned ? kThreads / 32 : 1][kLearned ? kDraws : 1];
    __shared__ unsigned long long s_stats[kMaxReq * kStats];
    const int tid = threadIdx.x, lane = tid & 31;
    constexpr bool learned = kLearned;
    unsigned char* wl = sw;
    unsigned char* wpth = sw + kBytesL;
    unsigned char* wev = sw + kBytesL + kBytesP;
    float* stage = s_stage[tid >> 5];
    float* draws = s_draws[kLearned ? tid >> 5 : 0];
    if constexpr (learned) {
        mmadec::stage_weights<kHalfBF16, 1, kSplit == 3>(wl, B.wL, 2 + kLatL, 1);
        mmadec::stage_weights<kHalfBF16, 2, kSplit == 3>(wpth, B.wP, 3 + kLatP, 3);
        mmadec::stage_weights<kHalfBF16, 2, kSplit == 3>(wev, B.wE, 7 + kLatE, 6);
    }
    for (int k = tid; k < kMaxReq * kStats; k += kThreads) s_stats[k] = 0ull;
    if (tid == 0) atomicMin(B.t_start, global_ns());
    __syncthreads();

    // counters of the lane's paths of request `req` (see flush_counters)
    constexpr int kCnt = kTimers ? kUsedStats + 1 : kUsedStats;   // + shadow-march steps (stats[11])
    unsigned cnt[kCnt];
#pragma unroll
    for (int j = 0; j < kCnt; ++j) cnt[j] = 0u;
    unsigned long long phase_cycles[4] = {0ull, 0ull, 0ull, 0ull};   // kTimers: march, decoder, transition, refill
    long long t_prev = kTimers ? clock64() : 0;
    int last_phase = -1;

    // ---- the lane's path ----
    int st = kIdle, req = 0, ev = 0;
    uint32_t id_lo = 0, id_hi = 0, seg = 0;
    V p = v3(0, 0, 0), w = v3(0, 0, 1);        // position and direction of the path
    float acc = 0.0f;                           // NEE sum of the path
    V nX = v3(0, 0, 0), nW = v3(0, 0, 1);       // pending NEE request
    float nwt = 0.0f;
    bool end_after = false;                     // the path ends after its pending NEE
    float u1 = 0.0f, u2 = 0.0f, u3 = 0.0f;      // this segment's HG cosine, azimuth and roulette uniforms
    float rad = 0.0f, tau = 0.0f;               // sphere of a parked (decode) lane
    // ---- the lane's current march ----
    V mo = v3(0, 0, 0), md = v3(0, 0, 1);
    float mt = 0.0f, ml = 0.0f, din = 0.0f;
    int mstep = 0;
    bool inside = true, capped = false;
    Geo geo{0.0f, 0.0f, 1.0f, 1.0f, 0.0f};
    bool drained = false;                       // warp-uniform: camera tickets exhausted

    // The lane's counters belong to request `req` and run over the lane's successive paths of that request; they
    // go into the block's counters when the lane takes a path of another request, when the largest nears 2^32,
    // and when the lane finishes.
    auto flush_counters = [&]() {
#pragma unroll
        for (int j = 0; j < kCnt; ++j) {
            if (cnt[j]) atomicAdd(&s_stats[req * kStats + (j < kUsedStats ? j : 11)], (unsigned long long)cnt[j]);
            cnt[j] = 0u;
        }
    };
    auto end_path = [&]() {
        const Req& qe = B.r[req];
        if (acc != 0.0f) atomicAdd(&B.image[qe.image_offset + id_hi], (double)acc);
        // the request's last path: record its completion time (ns after the first block started)
        const unsigned long long total_r = (unsigned long long)qe.W * qe.H * qe.spp;
        if (atomicAdd(&B.done[req], 1ull) + 1ull == total_r)
            atomicExch(&B.stats[req * kStats + 10], global_ns() - *((volatile unsigned long long*)B.t_start));
        st = kIdle;
    };
    auto start_shadow = [&]() {
        const Req& q = B.r[req];
        mo = nX;
        const V dl = v3(q.light[0], q.light[1], q.light[2]) - nX;
        ml = sqrt_approx(dot(dl, dl));
        md = dl * __fdividef(1.0f, ml);
        mt = 0.0f;
        din = 0.0f;
        inside = true;
        capped = false;
        mstep = 0;
        st = kShadow;
    };

    for (;;) {
        if constexpr (kTimers) {
            const long long now = clock64();
            if (last_phase >= 0) phase_cycles[last_phase] += (unsigned long long)(now - t_prev);
            t_prev = now;
        }
        unsigned idle = __ballot_sync(0xffffffffu, st == kIdle);
        unsigned marching = __ballot_sync(0xffffffffu, st >= kCamera && st <= kShadow);
        // ---------------- refill round: new camera samples for idle lanes ----------------
        if (idle && !drained && (__popc(idle) >= kRefillBatch || __popc(marching) < 16)) {
            last_phase = 3;
            const int leader = __ffs(idle) - 1;
            unsigned long long t0 = 0;
            if (lane == leader) t0 = atomicAdd(B.ticket, (unsigned long long)__popc(idle));
            t0 = __shfl_sync(0xffffffffu, t0, leader);
            if (t0 + __popc(idle) >= B.total) drained = true;
            const uint64_t t = t0 + __popc(idle & ((1u << lane) - 1u));
            if (st == kIdle && t < B.total) {
                const int nreq = find_req(B, t);
                if (nreq != req || cnt[8] > (1u << 30)) flush_counters();
                req = nreq;
                const Req& q = B.r[req];
                const uint64_t local = t - q.samples_begin;
                if ((local >> 32) == 0) {                         // the usual case: 32-bit division
                    id_hi = (uint32_t)local / q.spp;
                    id_lo = (uint32_t)q.sample_offset + ((uint32_t)local - id_hi * q.spp);
                } else {
                    id_hi = (uint32_t)(local / q.spp);
                    id_lo = (uint32_t)(q.sample_offset + local % q.spp);
                }
                const Stream rs(q.seed, ((uint64_t)id_hi << 32) | id_lo);
                const Words j = rs.at(0u, 8u);
                camera_ray(q, (int)(id_hi % (uint32_t)q.W), (int)(id_hi / (uint32_t)q.W), u24(j.w0), u24(j.w1),
                           &mo, &md);
                seg = 0;
                acc = 0.0f;
                end_after = false;
                mt = 0.0f;
                mstep = 0;
                st = kCamera;
                geo = Geo{q.A, q.k, q.inv_lip, q.rb2, q.din_cut};
                cnt[0] += 1u;
            }
            continue;
        }
        const unsigned parked = __ballot_sync(0xffffffffu, st == kDecode);
        const unsigned pending = __ballot_sync(0xffffffffu, st == kPending);
        if (!parked && !pending && !marching) break;   // drained and no lane holds a path
        const int n_active = __popc(marching);

        if (learned && parked && (__popc(parked) >= kDecodeBatch || n_active + __popc(pending) < kDecodeBatch)) {
            // ================= decoder round: the three learned samplers for the parked lanes =================
            last_phase = 1;
            // The first 16 parked lanes (by lane index) are compacted into the 16 rows of one tensor-core tile;
            // the MLPs run on that tile (in the decoders' precision, kDec), and lanes parked beyond it wait for the
            // next round.  Everything else per path stays in the lane's registers.
            const int rank = __popc(parked & ((1u << lane) - 1u));
            const bool mine = st == kDecode && rank < 16;
            const Req& qq = B.r[req];
            // The step's draws (tags 2..7: 24 normals; the low bytes of words 0..2 of tags 2..6, unused by the
            // normals, give the absorption, azimuth, exact-N = 1, centre-event and N = 1 exit uniforms) are the
            // same Philox blocks as drawn lane by lane, but the 6 blocks of each of the nsel selected paths are
            // spread over all 32 lanes and handed over through shared memory: value v of row r at
            // draws[v * 16 + r].
            const int nsel = min(16, __popc(parked));
            uint32_t* keys = reinterpret_cast<uint32_t*>(stage) + kDrawKeys;
            if (mine) {
                keys[5 * rank] = id_lo;
                keys[5 * rank + 1] = id_hi;
                keys[5 * rank + 2] = seg;
                keys[5 * rank + 3] = (uint32_t)qq.seed;
                keys[5 * rank + 4] = (uint32_t)(qq.seed >> 32);
            }
            __syncwarp();
#pragma unroll 1
            for (int i = lane; i < 6 * nsel; i += 32) {
                const int c = (int)__fdividef((float)i + 0.5f, (float)nsel);   // block c (tag 2 + c) of row r
                const int r = i - c * nsel;
                const uint32_t* kr = keys + 5 * r;
                const Words wd = philox(kr[2], kr[0], kr[1], 2u + (uint32_t)c, kr[3], kr[4]);
                const float2 a = box_muller(wd.w0, wd.w1), b = box_muller(wd.w2, wd.w3);
                float* o = draws + 4 * c * 16 + r;
                o[0] = a.x; o[16] = a.y; o[32] = b.x; o[48] = b.y;
                if (c < 5)
                    draws[(24 + c) * 16 + r] =
                        (float)(((wd.w0 & 0xffu) << 16) | ((wd.w1 & 0xffu) << 8) | (wd.w2 & 0xffu)) * 0x1.0p-24f;
            }
            __syncwarp();
            // the row's draws are read where they are used (they stay in shared memory, not in registers)
            const int rr = mine ? rank : 0;
            auto nrm = [&](int v) -> float { return draws[v * 16 + rr]; };
            float ltau = 0.0f;
            if (mine) {
                cnt[3] += 1u;
                ltau = __logf(tau);
            }
            // LengthGen: N (albedo-1 physics, Eq. 3)
            float xin[16] = {ltau, mine ? qq.g : 0.0f, nrm(kZL), nrm(kZL + 1)};
            float yL[8];
            mmadec::warp_mlp_rows16<1, kSplit, kHalfBF16, 1, 2 + kLatL, 2>(wl, stage, xin, yL, rank, mine);
            const float yN = yL[0] + __expf(0.5f * yL[1]) * nrm(kEL);
            float N = floorf(__expf(yN) + 0.5f);
            N = fminf(fmaxf(N, mine && qq.exact_n1 ? 2.0f : 1.0f), kNMax);
            // exact_n1: N = 1 (the first free path from the centre leaves the sphere) drawn with its exact
            // probability exp(-tau), LengthGen (trained on the N >= 2 records) giving the rest; such a step is
            // exact as a whole (exit along the centre event's HG direction, that event the representative one)
            if (mine && qq.exact_n1 && nrm(26) < __expf(-tau)) N = 1.0f;
            const bool one = mine && qq.exact_n1 && N <= 1.0f;
            const float lnN = mine ? __logf(N) : 0.0f;
            // PathGen: (cos theta, alpha, beta)
            float xp[16] = {ltau, mine ? qq.g : 0.0f, lnN, nrm(kZP), nrm(kZP + 1), nrm(kZP + 2), nrm(kZP + 3),
                            nrm(kZP + 4)};
            float yP[8];
            mmadec::warp_mlp_rows16<1, kSplit, kHalfBF16, 2, 3 + kLatP, 6>(wpth, stage, xp, yP, rank, mine);
            float ct = fminf(1.0f, fmaxf(-1.0f, yP[0] + __expf(0.5f * yP[3]) * nrm(kEP)));
            float al = yP[1] + __expf(0.5f * yP[4]) * nrm(kEP + 1);
            float be = yP[2] + __expf(0.5f * yP[5]) * nrm(kEP + 2);
            float ab2 = al * al + be * be;
            if (ab2 > 1.0f) {
                const float s = rsqrtf(ab2);
                al *= s; be *= s; ab2 = 1.0f;
            }
            // EventGen: representative event (X~, W~)
            float xe[16] = {ltau, mine ? qq.g : 0.0f, mine ? qq.phi : 0.0f, ct, al, be, lnN,
                            nrm(kZE), nrm(kZE + 1), nrm(kZE + 2), nrm(kZE + 3), nrm(kZE + 4)};
            float yE[16];
            mmadec::warp_mlp_rows16<2, kSplit, kHalfBF16, 2, 16, 12>(wev, stage, xe, yE, rank, mine);
            if (mine) {
                float e[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) e[k] = yE[k] + __expf(0.5f * yE[6 + k]) * nrm(kEE + k);
                if (one) {
                    ct = hg_cosine(nrm(28), qq.g);
                    al = be = ab2 = 0.0f;
                }
                const float phiN = __expf(N * qq.log_phi);
                const float lam = qq.phi < 1.0f ? __fdividef(qq.phi * (1.0f - phiN), 1.0f - qq.phi) : N;
                // exact_centre: the first event (the centre, incoming direction) is the representative one with
                // probability phi / Lambda (Sec. 4.3, k = 1), drawn as such; EventGen gives the later ones
                // (and exact_n1's N = 1 step takes the centre too)
                if (N <= 1.0f ? (qq.exact_n1 || qq.exact_centre)
                              : (qq.exact_centre && nrm(27) < __fdividef(qq.phi, lam))) {
                    e[0] = e[1] = e[2] = 0.0f;
                    e[3] = e[4] = 0.0f;
                    e[5] = 1.0f;
                }
                // Eq. 4 and Sec. 4.1: CVAE frame -> world via R^CVAE R_psi, scaled by r
                V t1, t2;
                onb(w, &t1, &t2);
                float sn, cs;
                sincos_turns_fast(nrm(25), &sn, &cs);
                const float stt = sqrt_approx(fmaxf(0.0f, 1.0f - ct * ct));
                const float nn = sqrt_approx(fmaxf(0.0f, 1.0f - ab2));
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
                    vw[k] = t1 * v1.x + t2 * v1.y + w * v1.z;
                }
                nX = p + vw[2] * rad;                   // p holds the collision point c
                nW = unit(vw[3]);
                nwt = lam;
                if (nrm(24) >= phiN) {
                    cnt[5] += 1u;
                    end_after = true;
                } else {
                    const V xexit = p + vw[0] * rad;
                    w = unit(vw[1]);
                    p = xexit;
                    seg += 1u;
                }
                start_shadow();
            }
            continue;
        }

        if (pending && (__popc(pending) >= kTransBatch || n_active < 16)) {
            // ================= transition round: what follows each finished march =================
            last_phase = 2;
            if (st == kPending) {
                const Req& q = B.r[req];
                bool need_flight = false, finish = false;   // one end_path call site for the whole round
                if (ev == kEvShadowDone) {
                    cnt[7] += 1u;
                    if (capped) {
                        cnt[6] += 1u;
                    } else {
                        const float rho = hg_pdf(dot(nW, md), q.g);
                        acc += __fdividef(nwt * rho * __expf(-q.sigma * din) * q.I, ml * ml);
                    }
                    finish = end_after;
                    need_flight = !end_after;
                } else if (ev == kEvCollide) {
                    const V c = mo + md * ml;
                    bool sphere = false;
                    if (q.mode == MS_SPHERE && learned) {
                        float dc = -sdf(geo, c) * geo.inv_lip;
                        if (q.grid) {
                            // the voxel holding c: its value bounds the distance from every point of the voxel
                            const int n1 = q.grid_n - 1;
                            const int ix = min(max((int)((c.x + q.grid_b) * q.grid_inv_h), 0), n1);
                            const int iy = min(max((int)((c.y + q.grid_b) * q.grid_inv_h), 0), n1);
                            const int iz = min(max((int)((c.z + q.grid_b) * q.grid_inv_h), 0), n1);
                            dc = fmaxf(dc, __ldg(q.grid + ((size_t)iz * q.grid_n + iy) * q.grid_n + ix));
                        }
                        cnt[8] += 1u;
                        rad = fminf(dc, q.tau_max * q.inv_sigma);
                        tau = q.sigma * rad;
                        if (tau >= q.tau_min) {
                            sphere = true;
                            p = c;
                            st = kDecode;                // park until the warp runs a decoder round
                        }
                    }
                    if (!sphere) {
                        // brute-force event: NEE at c with weight phi, roulette, HG scattering (Sec. 3.1)
                        cnt[4] += 1u;
                        nX = c;
                        nW = md;
                        nwt = q.phi;
                        if (u3 >= q.phi) {
                            cnt[5] += 1u;
                            end_after = true;
                        } else {
                            w = scatter_dir(md, hg_cosine(u1, q.g), u2);
                            p = c;
                            seg += 1u;
                        }
                        start_shadow();
                    }
                } else if (ev == kEvExit) {
                    st = kReentry;                       // left the object at mo: look for a re-entry
                    mt = 0.0f;
                    mstep = 0;
                } else if (ev == kEvHit || ev == kEvReenter) {
                    need_flight = true;
                } else {
                    if (ev == kEvCap) cnt[6] += 1u;
                    finish = true;
                }
                if (need_flight) {
                    if (seg >= q.max_segments) {
                        cnt[6] += 1u;
                        finish = true;
                    } else {
                        cnt[2] += 1u;
                        const Stream rs(q.seed, ((uint64_t)id_hi << 32) | id_lo);
                        const Words u = rs.at(seg, 0u);
                        ml = -__logf(1.0f - u24(u.w0)) * q.inv_sigma;
                        u1 = u24(u.w1);
                        u2 = u24(u.w2);
                        u3 = u24(u.w3);
                        mo = p;
                        md = w;
                        mt = 0.0f;
                        mstep = 0;
                        st = kFlight;
                    }
                }
                if (finish) end_path();
            }
            continue;
        }

        // ================= kSteps signed-distance steps of every marching lane =================
        last_phase = 0;
        // One body for every kind of march (selects, no per-kind branches), so lanes in different kinds of
        // march stay converged; only boundary crossings, which are rare, branch.
#pragma unroll 1
        for (int step = 0; step < kSteps; ++step) {
            // the round ends early once no lane marches (its marches are short: a few steps on average)
            if (!__any_sync(0xffffffffu, st >= kCamera && st <= kShadow)) break;
            if (st < kCamera || st > kShadow) continue;
            const V r = mo + md * mt;
            const bool shadow = st == kShadow, flight = st == kFlight;
            const bool in_medium = flight || (shadow && inside);
            // outside the medium the march ends when it leaves the bounding sphere (escape, or the rest of
            // a shadow segment); the end of a shadow segment is tested before the distance evaluation
            const bool leaving = !in_medium && dot(r, r) > geo.rb2 && dot(r, md) >= 0.0f;
            ++mstep;
            if ((shadow && mt >= ml) || leaving) {
                ev = shadow ? kEvShadowDone : kEvEscape;
                st = kPending;
                continue;
            }
            float rp, irp, R0, gd;
            const float f = sdf_parts_grad(geo, r, md, &rp, &irp, &R0, &gd);
            cnt[8] += 1u;
            if constexpr (kTimers) cnt[kCnt - 1] += shadow ? 1u : 0u;
            const float hs = in_medium ? -f : f, h1 = in_medium ? -gd : gd;   // the marched side's distance
            const float dl = hs * geo.inv_lip;
            // boundary band: the point is on the surface; the ray crosses there if it moves to the other side,
            // else steps off with the curvature step.  Elsewhere: the largest of the three steps.  (Selects,
            // not branches: most iterations hold lanes of both kinds.)
            const bool band = dl < kEps;
            cnt[9] += band ? 1u : 0u;
            const float cs = curve_step(geo, irp, rp, band ? fmaxf(hs, 0.0f) : hs, h1, in_medium);
            bool escape;
            const float ss = safe_step(geo, r, md, rp, R0, f, in_medium, &escape);
            const bool crossing = band && h1 < 0.0f;
            escape = escape && !band;
            float d = band ? fmaxf(kEps, cs) : fmaxf(fmaxf(dl, ss), cs);
            if (escape) {                                    // the surface is out of reach along the ray
                ev = shadow ? kEvShadowDone : kEvEscape;
                st = kPending;
                continue;
            }
            if (crossing) {
                if (shadow) {
                    inside = !inside;                        // same point, other side: no step
                    if (mstep >= kMaxMarch) { capped = true; ev = kEvShadowDone; st = kPending; }
                } else if (flight) {
                    mo = r;                                  // left the object at r
                    ev = kEvExit;
                    st = kPending;
                } else {
                    if (st == kCamera) {
                        cnt[1] += 1u;
                        w = md;
                        ev = kEvHit;
                    } else {
                        seg += 1u;
                        ev = kEvReenter;
                    }
                    p = r;
                    st = kPending;
                }
                continue;
            }
            // a flight ends at its free path, a shadow march at the light; outside marches have no limit
            const float lim = (flight || shadow) ? ml : 3.0e38f;
            const bool reach = mt + d >= lim;
            const float adv = reach ? lim - mt : d;
            if (shadow && inside) din += adv;
            mt += adv;
            // a shadow ray whose optical depth has passed kTauCut ends here: its transmittance is below
            // exp(-kTauCut) (about 1e-13) of the unshadowed term, and the rest of the segment can only lower it
            if (reach || (shadow && din > geo.din_cut)) {
                ev = flight ? kEvCollide : kEvShadowDone;
                st = kPending;
            } else if (mstep >= kMaxMarch) {
                capped = shadow;
                ev = shadow ? kEvShadowDone : kEvCap;
                st = kPending;
            }
        }
    }

    flush_counters();
    // ---------------- block counters -> global ----------------
    if constexpr (kTimers) {
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(&s_stats[12 + k], phase_cycles[k]);
    }
    __syncthreads();
    for (int k = tid; k < B.n * kStats; k += kThreads)
        if (s_stats[k]) atomicAdd(&B.stats[k], s_stats[k]);
}

// The compiled scheduling variants (decode batch, transition batch, most steps per march round, blocks per
// SM); index 0 is the default.  The sphere-tracing picks lie within 2% of each other on the four-density
// benchmark; brute force (no decoder rounds) prefers larger transition batches and longer march rounds (the last
// three).  A decoder round takes at most 16 parked lanes (one tensor-core tile), so the decode thresholds stay
// <= 16.
#define MS_RENDER_VARIANTS(X)                                                                                 \
    X(10, 12, 24, 3) X(8, 14, 28, 3) X(8, 12, 32, 3) X(12, 12, 24, 3) X(10, 14, 24, 3) X(10, 12, 28, 3)        \
    X(10, 16, 32, 3) X(10, 20, 32, 3) X(10, 16, 48, 3)

// The kernel of variant i with decoder arithmetic kDec (one translation unit per kDec, compiled in parallel).
template <int kDec>
const void* variant_kernel(int i)
{
    int k = 0;
    const void* fn = nullptr;
#define MS_RENDER_PICK(d, t, s, m)                                                                            \
    if (k++ == i) fn = (const void*)render_kernel<d, t, s, m, kDec>;
    MS_RENDER_VARIANTS(MS_RENDER_PICK)
#undef MS_RENDER_PICK
    return fn;
}
const void* variant_kernel_fp16(int i);    // render_f16.cu
const void* variant_kernel_bf16(int i);    // render_bf16.cu

}  // namespace render
}  // namespace ms
