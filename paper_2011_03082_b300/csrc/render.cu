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
//    registers flushed to shared, then global, memory;
//  * everything is bounded: segments per path, steps per march, and the loop ends when the ticket is drained
//    and no lane holds a path.
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

struct Req {
    float cam[3], at[3], tan_half, aspect;
    float light[3], I;
    float sigma, g, phi, log_phi, A, k, lip, inv_lip, rb2;
    float tau_min, tau_max;
    const float* grid;               // voxel grid of conservative distances, or null
    int32_t grid_n;
    float grid_b, grid_inv_h;
    int32_t W, H, mode;
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
    float A, k, inv_lip, rb2;
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
constexpr int kDraws = 26 * 16;      // a decoder round's draws: value v of row r at [v * 16 + r]
constexpr int kDrawKeys = 0;         // staging-tile offset of the draw keys (5 words per row) in a decoder round
static_assert(kDrawKeys + 5 * 16 <= mmadec::kStageFloats, "decoder-round draw keys exceed the staging tile");

// Scheduling constants of a kernel variant (see ms_render_autotune): kDecodeBatch parked lanes trigger a
// decoder round, kTransBatch pending (or idle) lanes a transition (or refill) round, and between two
// scheduling decisions each marching lane advances kSteps signed-distance steps.

enum State : int { kIdle = 0, kCamera, kFlight, kReentry, kShadow, kDecode, kPending };
enum Event : int { kEvHit = 0, kEvReenter, kEvEscape, kEvCap, kEvExit, kEvCollide, kEvShadowDone };

// kLearned: the launch holds at least one sphere-tracing request (decoder weights present); the brute-force
// instantiation carries no decoder code, which leaves its march and transitions free of register spills.
template <int kDecodeBatch, int kTransBatch, int kSteps, int kMinBlocks, bool kLearned>
__global__ void __launch_bounds__(kThreads, kMinBlocks) render_kernel(const __grid_constant__ Batch B)
{
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
        mmadec::stage_weights<false, 1>(wl, B.wL, 2 + kLatL, 1);
        mmadec::stage_weights<false, 2>(wpth, B.wP, 3 + kLatP, 3);
        mmadec::stage_weights<false, 2>(wev, B.wE, 7 + kLatE, 6);
    }
    for (int k = tid; k < kMaxReq * kStats; k += kThreads) s_stats[k] = 0ull;
    if (tid == 0) atomicMin(B.t_start, global_ns());
    __syncthreads();

    // counters of the lane's current path (flushed into its request's shared counters when the path ends)
    unsigned cnt[kUsedStats];
#pragma unroll
    for (int j = 0; j < kUsedStats; ++j) cnt[j] = 0u;

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
    Geo geo{0.0f, 0.0f, 1.0f, 1.0f};
    bool drained = false;                       // warp-uniform: camera tickets exhausted

    auto end_path = [&]() {
        const Req& qe = B.r[req];
        if (acc != 0.0f) atomicAdd(&B.image[qe.image_offset + id_hi], (double)acc);
        // the request's last path: record its completion time (ns after the first block started)
        const unsigned long long total_r = (unsigned long long)qe.W * qe.H * qe.spp;
        if (atomicAdd(&B.done[req], 1ull) + 1ull == total_r)
            atomicExch(&B.stats[req * kStats + 10], global_ns() - *((volatile unsigned long long*)B.t_start));
#pragma unroll
        for (int j = 0; j < kUsedStats; ++j) {
            if (cnt[j]) atomicAdd(&s_stats[req * kStats + j], (unsigned long long)cnt[j]);
            cnt[j] = 0u;
        }
        st = kIdle;
    };
    auto start_shadow = [&]() {
        const Req& q = B.r[req];
        mo = nX;
        const V dl = v3(q.light[0], q.light[1], q.light[2]) - nX;
        ml = sqrtf(dot(dl, dl));
        md = dl * (1.0f / ml);
        mt = 0.0f;
        din = 0.0f;
        inside = true;
        capped = false;
        mstep = 0;
        st = kShadow;
    };

    for (;;) {
        unsigned idle = __ballot_sync(0xffffffffu, st == kIdle);
        unsigned marching = __ballot_sync(0xffffffffu, st >= kCamera && st <= kShadow);
        // ---------------- refill round: new camera samples for idle lanes ----------------
        if (idle && !drained && (__popc(idle) >= kRefillBatch || __popc(marching) < 16)) {
            const int leader = __ffs(idle) - 1;
            unsigned long long t0 = 0;
            if (lane == leader) t0 = atomicAdd(B.ticket, (unsigned long long)__popc(idle));
            t0 = __shfl_sync(0xffffffffu, t0, leader);
            if (t0 + __popc(idle) >= B.total) drained = true;
            const uint64_t t = t0 + __popc(idle & ((1u << lane) - 1u));
            if (st == kIdle && t < B.total) {
                req = find_req(B, t);
                const Req& q = B.r[req];
                const uint64_t local = t - q.samples_begin;
                id_hi = (uint32_t)(local / q.spp);
                id_lo = (uint32_t)(q.sample_offset + local % q.spp);
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
                geo = Geo{q.A, q.k, q.inv_lip, q.rb2};
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
            // The first 16 parked lanes (by lane index) are compacted into the 16 rows of one tensor-core tile;
            // the MLPs run on that tile, and lanes parked beyond it wait for the next round.  Everything else
            // per path stays in the lane's registers.
            const int rank = __popc(parked & ((1u << lane) - 1u));
            const bool mine = st == kDecode && rank < 16;
            const Req& qq = B.r[req];
            // The step's draws (tags 2..7: 24 normals; the low bytes of words 0..2 of tags 2 and 3, unused by
            // the normals, give the absorption and azimuth uniforms) are the same Philox blocks as drawn lane
            // by lane, but the 6 blocks of each of the nsel selected paths are spread over all 32 lanes and
            // handed over through shared memory: value v of row r at draws[v * 16 + r].
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
                if (c < 2)
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
            mmadec::warp_mlp_rows16<1, 3, false, 1, 2 + kLatL, 2>(wl, stage, xin, yL, rank, mine);
            const float yN = yL[0] + __expf(0.5f * yL[1]) * nrm(kEL);
            float N = floorf(__expf(yN) + 0.5f);
            N = fminf(fmaxf(N, 1.0f), kNMax);
            const float lnN = mine ? __logf(N) : 0.0f;
            // PathGen: (cos theta, alpha, beta)
            float xp[16] = {ltau, mine ? qq.g : 0.0f, lnN, nrm(kZP), nrm(kZP + 1), nrm(kZP + 2), nrm(kZP + 3),
                            nrm(kZP + 4)};
            float yP[8];
            mmadec::warp_mlp_rows16<1, 3, false, 2, 3 + kLatP, 6>(wpth, stage, xp, yP, rank, mine);
            const float ct = fminf(1.0f, fmaxf(-1.0f, yP[0] + __expf(0.5f * yP[3]) * nrm(kEP)));
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
            mmadec::warp_mlp_rows16<2, 3, false, 2, 16, 12>(wev, stage, xe, yE, rank, mine);
            if (mine) {
                float e[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) e[k] = yE[k] + __expf(0.5f * yE[6 + k]) * nrm(kEE + k);
                const float phiN = __expf(N * qq.log_phi);
                const float lam = qq.phi < 1.0f ? qq.phi * (1.0f - phiN) / (1.0f - qq.phi) : N;
                // Eq. 4 and Sec. 4.1: CVAE frame -> world via R^CVAE R_psi, scaled by r
                V t1, t2;
                onb(w, &t1, &t2);
                float sn, cs;
                sincos_turns_fast(nrm(25), &sn, &cs);
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
            if (st == kPending) {
                const Req& q = B.r[req];
                bool need_flight = false, finish = false;   // one end_path call site for the whole round
                if (ev == kEvShadowDone) {
                    cnt[7] += 1u;
                    if (capped) {
                        cnt[6] += 1u;
                    } else {
                        const float rho = hg_pdf(dot(nW, md), q.g);
                        acc += nwt * rho * __expf(-q.sigma * din) * q.I / (ml * ml);
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
                        rad = fminf(dc, q.tau_max / q.sigma);
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
                        ml = -__logf(1.0f - u24(u.w0)) / q.sigma;
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
        // One body for every kind of march (selects, no per-kind branches), so lanes in different kinds of
        // march stay converged; only boundary crossings, which are rare, branch.
#pragma unroll 1
        for (int step = 0; step < kSteps; ++step) {
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
            if (reach) {
                ev = flight ? kEvCollide : kEvShadowDone;
                st = kPending;
            } else if (mstep >= kMaxMarch) {
                capped = shadow;
                ev = shadow ? kEvShadowDone : kEvCap;
                st = kPending;
            }
        }
    }

    // ---------------- block counters -> global ----------------
    __syncthreads();
    for (int k = tid; k < B.n * kStats; k += kThreads)
        if (s_stats[k]) atomicAdd(&B.stats[k], s_stats[k]);
}

}  // namespace render
}  // namespace ms

using namespace ms::render;

// Compiled kernel variants (scheduling constants); index 0, the one the autotuner usually selects on the
// four-density benchmark, is the default.
struct Variant {
    const void* fn;          // with the decoders (any sphere-tracing request)
    const void* fn_brute;    // brute force only
    int decode_batch, trans_batch, steps, min_blocks;
};
template <int D, int T, int S, int M>
Variant make_variant()
{
    return Variant{(const void*)render_kernel<D, T, S, M, true>, (const void*)render_kernel<D, T, S, M, false>, D, T, S, M};
}
// A decoder round takes at most 16 parked lanes (one tensor-core tile), so the decode thresholds stay <= 16.
static const Variant kVariants[] = {
    make_variant<10, 12, 24, 3>(), make_variant<12, 12, 24, 3>(), make_variant<8, 12, 24, 3>(),
    make_variant<10, 14, 24, 3>(), make_variant<10, 12, 20, 3>(), make_variant<10, 12, 28, 3>(),
    make_variant<10, 16, 24, 3>(), make_variant<10, 10, 28, 3>(), make_variant<8, 14, 28, 3>(),
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

static ms_status fill_batch(const ms_render_params* reqs, int n, Batch* b, const char* fn)
{
    if (n < 1 || n > kMaxReq) return ms::set_error(MS_ERR_INVALID_ARG, "%s: 1..%d requests per call", fn, kMaxReq);
    if (reqs[0].variant < 0 || reqs[0].variant >= kNumVariants)
        return ms::set_error(MS_ERR_INVALID_ARG, "%s: variant must be in 0..%d", fn, kNumVariants - 1);
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
        q.inv_lip = 1.0f / q.lip;
        const float rb = 1.0f + p.disp_amp + 1e-3f;
        q.rb2 = rb * rb;
        q.tau_min = p.min_optical_radius;
        q.tau_max = p.max_optical_radius;
        if (p.sdf_grid != nullptr) {
            if (p.sdf_grid_n < 4 || p.sdf_grid_n > 1024 || !(p.disp_amp < 1.0f))
                return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: sdf_grid_n must be in 4..1024", fn, i);
            const float h = 2.0f * (1.0f + p.disp_amp) / (float)(p.sdf_grid_n - 2);
            q.grid = p.sdf_grid;
            q.grid_n = p.sdf_grid_n;
            q.grid_b = 1.0f + p.disp_amp + h;
            q.grid_inv_h = 1.0f / h;
        } else {
            q.grid = nullptr;
            q.grid_n = 0;
            q.grid_b = q.grid_inv_h = 0.0f;
        }
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
    return 1024;   // ticket, start time, finished-path counters of up to 64 requests
}

static ms_status render_launch(const ms_render_params* reqs, int n, const ms_cvae_set* models, double* images,
                               unsigned long long* stats, void* workspace, size_t workspace_bytes, void* stream,
                               const char* fn)
{
    MS_CHECK_ARG(reqs != nullptr && images != nullptr && stats != nullptr, "%s: null argument", fn);
    const size_t need_ws = ms_render_workspace_size(reqs, n);
    MS_CHECK_ARG(workspace != nullptr && workspace_bytes >= need_ws && ((uintptr_t)workspace & 255u) == 0,
                 "%s: a 256-byte aligned workspace of at least %zu bytes is required", fn, need_ws);
    Batch b;
    ms_status st = fill_batch(reqs, n, &b, fn);
    if (st != MS_OK) return st;
    bool any_sphere = false;
    for (int i = 0; i < n; ++i) any_sphere |= reqs[i].mode == MS_SPHERE;
    b.wL = b.wP = b.wE = nullptr;
    if (any_sphere) {
        MS_CHECK_ARG(models != nullptr, "%s: MS_SPHERE needs the three decoders", fn);
        const ms_decoder* d[3] = {&models->length, &models->path, &models->event};
        const int pin[3] = {2, 3, 7}, pout[3] = {1, 3, 6}, lat[3] = {kLatL, kLatP, kLatE}, wid[3] = {8, 16, 16};
        for (int k = 0; k < 3; ++k) {
            MS_CHECK_ARG(d[k]->weights != nullptr && d[k]->p_in == pin[k] && d[k]->p_out == pout[k] &&
                             d[k]->latent == lat[k] && d[k]->width == wid[k],
                         "%s: decoder %d must have p_in %d, latent %d, width %d, p_out %d (Table 1)", fn, k, pin[k],
                         lat[k], wid[k], pout[k]);
            MS_CHECK_ARG(d[k]->precision == MS_FP32, "%s: the renderer evaluates FP32 decoders", fn);
        }
        b.wL = models->length.weights;
        b.wP = models->path.weights;
        b.wE = models->event.weights;
    }
    b.image = images;
    b.stats = stats;
    b.ticket = static_cast<unsigned long long*>(workspace);
    b.t_start = b.ticket + 1;
    b.done = b.ticket + 2;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MS_CUDA(cudaMemsetAsync(workspace, 0, (2 + kMaxReq) * sizeof(unsigned long long), s));
    MS_CUDA(cudaMemsetAsync(b.t_start, 0xff, sizeof(unsigned long long), s));
    const Variant& v = kVariants[reqs[0].variant];
    const void* kfn = any_sphere ? v.fn : v.fn_brute;
    int per_sm = 0;
    MS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, 0));
    uint64_t grid = (uint64_t)ms::num_sms() * (per_sm > 0 ? per_sm : 1);
    const uint64_t need = (b.total + kThreads - 1) / kThreads;
    if (grid > need) grid = need;
    void* args[] = {&b};
    MS_CUDA(cudaLaunchKernel(kfn, dim3((unsigned)grid), dim3(kThreads), args, 0, s));
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

extern "C" int ms_render_variants(void) { return kNumVariants; }

extern "C" ms_status ms_render_variant_info(int i, int* decode_batch, int* trans_batch, int* steps, int* min_blocks)
{
    MS_CHECK_ARG(i >= 0 && i < kNumVariants, "ms_render_variant_info: variant must be in 0..%d", kNumVariants - 1);
    if (decode_batch) *decode_batch = kVariants[i].decode_batch;
    if (trans_batch) *trans_batch = kVariants[i].trans_batch;
    if (steps) *steps = kVariants[i].steps;
    if (min_blocks) *min_blocks = kVariants[i].min_blocks;
    return MS_OK;
}

extern "C" ms_status ms_render_autotune(const ms_render_params* reqs, int n, const ms_cvae_set* models, double* images,
                                        unsigned long long* stats, void* workspace, size_t workspace_bytes,
                                        int repeats, int* best_variant, float* ms_per_variant, void* stream)
{
    MS_CHECK_ARG(reqs != nullptr && n >= 1 && n <= kMaxReq && best_variant != nullptr,
                 "ms_render_autotune: need 1..%d requests and best_variant", kMaxReq);
    MS_CHECK_ARG(repeats >= 1, "ms_render_autotune: repeats must be >= 1");
    ms_render_params local[kMaxReq];
    for (int i = 0; i < n; ++i) local[i] = reqs[i];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    MS_CUDA(cudaEventCreate(&e0));
    MS_CUDA(cudaEventCreate(&e1));
    float best = 0.0f;
    int best_i = -1;
    ms_status st = MS_OK;
    for (int v = 0; v < kNumVariants && st == MS_OK; ++v) {
        local[0].variant = v;
        st = render_launch(local, n, models, images, stats, workspace, workspace_bytes, stream, "ms_render_autotune");
        if (st != MS_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < repeats && st == MS_OK; ++r)
            st = render_launch(local, n, models, images, stats, workspace, workspace_bytes, stream, "ms_render_autotune");
        cudaEventRecord(e1, s);
        if (st != MS_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = ms::cuda_status(cudaGetLastError(), "ms_render_autotune: cudaEventSynchronize");
            break;
        }
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        t /= (float)repeats;
        if (ms_per_variant) ms_per_variant[v] = t;
        if (best_i < 0 || t < best) {
            best = t;
            best_i = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == MS_OK) *best_variant = best_i;
    return st;
}
