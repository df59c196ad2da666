/*
 * ms.h — C ABI of the learned sphere-tracing library for subsurface scattering (one B300, sm_103a).
 *
 * The method (Leonard, Hoehlein, Westermann, "Learning Multiple-Scattering Solutions for Sphere-Tracing of
 * Volumetric Subsurface Effects"): light paths through a homogeneous translucent medium (extinction
 * sigma_t, albedo phi, Henyey-Greenstein anisotropy g) are advanced in large steps; at each collision the
 * largest sphere inside the boundary is taken from a signed distance function and three conditional-VAE
 * decoders sample what happens inside it: the number of scattering events N (LengthGen, which sets the
 * absorption probability 1 - phi^N), the exit point and direction (PathGen) and one representative
 * in-scatter event for next-event estimation (EventGen).  The brute-force Henyey-Greenstein walk is both the
 * plain method and the generator of the models' training data.
 *
 * Conventions for every entry point:
 *  - Pointers documented as "device" are CUDA device pointers owned by the caller; "host" pointers are read
 *    during the call only.  The library allocates no device memory: scratch space is passed in by the
 *    caller, sized by the matching *_workspace_size() function, and must be 256-byte aligned.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL means the legacy default stream);
 *    the call returns before the GPU finishes.  Outputs documented as "accumulated" are added to, so calls
 *    on disjoint photon or sample ranges (photon_offset, sample_offset) compose; the caller zeroes them.
 *  - Arguments passed by value or in host structs are validated on the host before anything is enqueued.
 *    Errors return a negative ms_status and leave a message for ms_last_error() (per host thread); no
 *    exception crosses the ABI.  A call that returns an error has enqueued nothing.  Values the caller keeps
 *    in device memory (per-photon media, weights, training data) are not read by the host and are not
 *    validated; out-of-range values there give meaningless results but cannot fault: every device loop has a
 *    cap and every histogram or voxel index is clamped.
 *  - Caps that are reached (events per photon, segments per path, steps per march) are counted in the
 *    asynchronous counters of the call (walk counters[2], render stats[6]); they are not return codes,
 *    because every call returns before the GPU finishes.
 *  - Random numbers come from the counter-based generator Philox4x32-10 keyed by `seed`; results depend only
 *    on (seed, ids, offsets) and not on launch configuration.
 */
#ifndef MS_H
#define MS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MS_OK = 0,
    MS_ERR_INVALID_ARG = -1,
    MS_ERR_CUDA = -2,           /* a CUDA runtime call failed; ms_last_error() has the CUDA error string   */
    MS_ERR_UNSUPPORTED = -4     /* unsupported shape or precision                                         */
} ms_status;

enum { MS_FP32 = 0, MS_FP64 = 1, MS_FP16 = 2, MS_BF16 = 3 };
enum { MS_BRUTE = 0, MS_SPHERE = 1 };
enum { MS_ESCAPED = 0, MS_ABSORBED = 1, MS_TRUNCATED = 2 };

/* Message of the last error on the calling host thread ("" if none). */
const char* ms_last_error(void);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int ms_version(void);

/* ------------------------------------------------------------------------------------------------------
 * Brute-force Henyey-Greenstein random walk in the unit sphere (Sec. 3.1, Eq. 1; reservoir Sec. 4.3).
 *
 * A photon starts at the centre with direction dir_in (or isotropic).  With first_event_at_origin = 1 (the
 * paper's training convention) the first scattering event is at the centre; with 0 the photon first flies.
 * Free paths are l = -log(1 - xi) / sigma_t with sigma_t the optical radius (sphere radius 1); at each event
 * Russian roulette continues with probability albedo and the new direction is drawn from the HG phase
 * function (cosine between old and new propagation direction, mean g); the walk ends at the first crossing
 * of the sphere.  N counts events including the one at the centre; an absorbed photon's N is the event at
 * which it was absorbed.  Random numbers of photon id at step s come from Philox4x32-10 counter
 * (s, id_lo, id_hi, tag) under key seed: tag 0 gives the free path, HG cosine, azimuth and roulette uniforms
 * (MS_FP32: word >> 8 as 24-bit uniforms; MS_FP64: 53-bit uniforms with the tag 2 words as low bits), and the
 * bits those leave unused give the reservoir's uniform (MS_FP32: the low bytes of words 0..2; MS_FP64: the low
 * 11 bits of the tag 2 words 0..2); tag 1 (and 3) at step 0 gives an isotropic start with an event at the
 * centre.
 * ---------------------------------------------------------------------------------------------------- */
typedef struct {
    float optical_radius;       /* sigma_t * R > 0                                  */
    float g;                    /* HG anisotropy, |g| < 1                            */
    float albedo;               /* phi in [0, 1]                                     */
    float dir_in[3];            /* incoming direction (normalised by the library)    */
    int32_t isotropic_start;    /* 1: initial direction uniform on the sphere        */
    int32_t first_event_at_origin;
} ms_medium;                    /* 32 bytes */

typedef struct {
    uint64_t seed;
    uint64_t photon_offset;     /* first photon id (for sharding)                                     */
    uint64_t n_photons;
    const ms_medium* media;     /* device: 1 entry, or n_photons entries if per_photon_media          */
    int32_t per_photon_media;
    uint32_t max_events;        /* a photon with this many events and no exit is truncated (>= 1)     */
    int32_t reservoir;          /* representative event: 0 none; 1 uniform over the events; 2 weights
                                   albedo^k with roulette off (training data: the path follows the
                                   albedo-1 physics, Sec. 3.2, and the event is chosen as in Sec. 4.3) */
    int32_t precision;          /* MS_FP32: 24-bit uniforms, single precision, the fast path.
                                   MS_FP64: 53-bit uniforms and double precision built from correctly
                                   rounded basic operations: every integer output is reproducible bit
                                   for bit by an implementation of the same steps.                     */
} ms_walk_params;

typedef struct {
    /* per photon, device, optional (NULL): indexed by photon id - photon_offset */
    int32_t* n_events;
    uint8_t* status;            /* MS_ESCAPED / MS_ABSORBED / MS_TRUNCATED                             */
    float* exit_pos;            /* [n][3] exit point on the unit sphere (0 if not escaped)             */
    float* exit_dir;            /* [n][3] exit direction (0 if not escaped)                            */
    float* rep_pos;             /* [n][3] representative event position (reservoir != 0)               */
    float* rep_dir;             /* [n][3] direction arriving at the representative event               */
    int32_t* rep_index;         /* [n] its event index k in 1..N (0: none)                             */
    /* accumulated, device, optional (NULL) */
    unsigned long long* hist_n;     /* [64]: bin 0 for N = 0, else min(63, 1 + 4*floor(log2 N) + the two
                                       bits below the leading one of N) — quarter octaves              */
    unsigned long long* hist_pos;   /* [32][64] escaped photons: cos(theta) = x_z in 32 equal bins over
                                       [-1,1], azimuth atan2(x_y, x_x) + pi in 64 equal bins          */
    unsigned long long* hist_cos;   /* [64] escaped photons: exit_dir . exit_pos in 64 bins over [0,1]  */
    unsigned long long* counters;   /* [8]: escaped, absorbed, truncated, total events, 0, 0, 0, 0     */
} ms_walk_out;

size_t ms_walk_workspace_size(const ms_walk_params* p);
/* Truncated photons are counted in counters[2]; the call does not wait for the GPU, so it returns MS_OK
 * and the caller reads the counters.  The media are device memory and are not validated (see the
 * conventions above): the ranges in ms_medium are the caller's to respect. */
ms_status ms_simulate_walks(const ms_walk_params* p, const ms_walk_out* out, void* workspace,
                            size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------------------------------------
 * Conditional-VAE decoder inference (Sec. 3.2): y = W3 sp(W2 sp(W1 [c; z] + b1) + b2) + b3 with
 * sp = Softplus, y = (mu, log Sigma) of a diagonal Gaussian, sample x = mu + exp(log Sigma / 2) * eps.
 * ---------------------------------------------------------------------------------------------------- */
typedef struct {
    int32_t p_in;               /* condition size, 1..12                                               */
    int32_t latent;             /* latent size L, 1..8 (p_in + latent <= 16)                          */
    int32_t width;              /* hidden width W, 8 or 16                                             */
    int32_t p_out;              /* output size P, 1..8                                                 */
    int32_t precision;          /* all on the tensor cores with FP32 accumulation.  MS_FP32: weights and
                                   activations split into FP16 head + tail, three products per tile
                                   (single-precision results, max |error| <= 1e-5); MS_FP16 / MS_BF16:
                                   weights rounded to FP16 / BF16, activations carried as two halves  */
    const float* weights;       /* device, packed float32: W1[W][p_in+L] b1[W] W2[W][W] b2[W]
                                   W3[2P][W] b3[2P] (row-major [out][in])                              */
} ms_decoder;

/* cond: device [n][p_in].  z_eps: device [n][latent + p_out] standard normals (z then eps), or NULL to draw
 * them in the kernel from query q's Philox blocks j = 0..B-1, counter (j, id_lo, id_hi, 0xD0), id = offset+q:
 * with c = latent + p_out normals, B is the fewest blocks with 4B + floor(4B/3) >= 2 ceil(c/2); uniform k < 4B
 * is the top 24 bits of word k (block k/4, word k%4), uniform 4B+i is the low bytes of words 3i, 3i+1, 3i+2
 * ((b0 << 16 | b1 << 8 | b2) 2^-24), and normals 2m, 2m+1 are Box-Muller on uniforms 2m, 2m+1.
 * out_mean_logvar: device [n][2P] or NULL; out_sample: device [n][P] or NULL. */
ms_status ms_cvae_infer(const ms_decoder* d, const float* cond, const float* z_eps, uint64_t seed,
                        uint64_t offset, uint64_t n, float* out_mean_logvar, float* out_sample, void* stream);

/* ------------------------------------------------------------------------------------------------------
 * CVAE training (Sec. 3.2): encoder Enc([x; c]) -> (mu_e, log Sigma_e) in R^L, z = mu_e + exp(lv_e/2) eps,
 * decoder as above; loss = mean over the batch of the negative ELBO
 *   0.5 sum_d (lv_d + (x_d - mu_d)^2 exp(-lv_d) + ln 2pi) + 0.5 sum_l (mu_l^2 + exp(lv_l) - lv_l - 1).
 * Parameters: encoder block E1[W][P+p_in] e1 E2[W][W] e2 E3[2L][W] e3, then the decoder block (as
 * ms_decoder.weights).  The optimiser is Adam (AdamW with weight_decay > 0), as in Sec. 3.2.
 * ---------------------------------------------------------------------------------------------------- */
typedef struct {
    int32_t p_in, p_out, latent, width;   /* a compiled shape: (p_in, p_out) in {(1,1) (2,1) (3,3) (4,1)
                                             (4,3) (4,6) (7,6)} with latent 4, width 16, or the Table 1
                                             shapes (2,1) latent 2 width 8, (3,3) and (7,6) latent 5
                                             width 16; MS_ERR_UNSUPPORTED otherwise                    */
    int32_t precision;                    /* MS_FP32 (BF16 compute with FP32 master weights: MS_BF16)   */
} ms_cvae_shape;

size_t ms_cvae_num_params(const ms_cvae_shape* s);
size_t ms_cvae_workspace_size(const ms_cvae_shape* s, uint64_t batch);

/* Loss and gradient of one batch.  x: device [B][p_out]; c: device [B][p_in]; eps_z: device [B][latent]
 * standard normals, or NULL to draw them: normals 4j..4j+3 of sample b come from counter
 * (j, b, step, 0xE0) by Box-Muller on 24-bit uniforms (B < 2^32).
 * grad: device [n_params] (overwritten) or NULL; loss3: device [3] (overwritten): loss, rec, kl.
 * The gradient reduction is deterministic (fixed order). */
ms_status ms_cvae_forward_backward(const ms_cvae_shape* s, const float* params, const float* x, const float* c,
                                   const float* eps_z, uint64_t B, uint64_t seed, uint64_t step, float* grad,
                                   float* loss3, void* workspace, size_t workspace_bytes, void* stream);

/* The loss alone (no gradient): loss3 (device [3], overwritten) = loss, rec, kl of the batch, from the same
 * forward pass, normals and fixed-order reduction as ms_cvae_forward_backward (equal to its loss3 bit for
 * bit).  Workspace as for ms_cvae_forward_backward.  The forward half of the torch.autograd.Function. */
ms_status ms_cvae_forward(const ms_cvae_shape* s, const float* params, const float* x, const float* c,
                          const float* eps_z, uint64_t B, uint64_t seed, uint64_t step, float* loss3,
                          void* workspace, size_t workspace_bytes, void* stream);

/* One bias-corrected Adam step t >= 1 on n parameters (device arrays, in place). */
ms_status ms_adam_step(float* params, float* m, float* v, const float* grad, uint64_t n, uint64_t t, float lr,
                       float beta1, float beta2, float eps, float weight_decay, void* stream);

/* ms_cvae_forward_backward followed by ms_adam_step (beta 0.9/0.999, eps 1e-8) on the same stream;
 * the gradient lives in the workspace. */
ms_status ms_cvae_train_step(const ms_cvae_shape* s, float* params, float* m, float* v, const float* x,
                             const float* c, const float* eps_z, uint64_t B, uint64_t seed, uint64_t step,
                             float lr, float weight_decay, float* loss3, void* workspace,
                             size_t workspace_bytes, void* stream);

/* A training step whose every input lives on the device, so that one captured CUDA graph can be replayed
 * step after step: `step` (device, the Adam step t >= 1) is read by the kernels and incremented at the end.
 * The mini-batch is drawn with replacement from the n_records records (x_all [n][p_out], c_all [n][p_in]):
 * sample b of step t takes record (w * n_records) >> 32, w = word 0 of counter (t_hi, t_lo, b, 0xB0) under
 * key seed; its latent normals come from counter (0, b, t, 0xE0) as in ms_cvae_forward_backward.  Adam
 * uses beta 0.9 / 0.999 and eps 1e-8 with bias corrections 1 - beta^t computed on the device. */
size_t ms_cvae_train_step_dev_workspace_size(const ms_cvae_shape* s, uint64_t batch);
ms_status ms_cvae_train_step_dev(const ms_cvae_shape* s, float* params, float* m, float* v, const float* x_all,
                                 const float* c_all, uint64_t n_records, uint64_t B, uint64_t seed,
                                 unsigned long long* step, float lr, float weight_decay, float* loss3,
                                 void* workspace, size_t workspace_bytes, void* stream);

/* The same training step with no workspace argument: its scratch is a fixed 16 MiB array inside the library
 * (ms_cvae_static_scratch_bytes()), for callers that must not allocate device memory — for example code whose
 * device memory is all owned by another framework's pool, or a plug-in that may not allocate while the host
 * application runs.  The paper has no counterpart; this is a deployment convenience.
 *  - Batches whose ms_cvae_workspace_size() exceeds the array are rejected with MS_ERR_INVALID_ARG.
 *  - Nothing is allocated, by this library or anything it calls.
 *  - Every device that loads the library keeps the array until the process exits.
 *  - All calls share the array: calls whose work overlaps on the GPU race and corrupt each other's
 *    gradients.  Nothing in it needs clearing between calls (each call overwrites what it reads).
 *  - The first call on a device looks the array's device address up (cudaGetSymbolAddress) and keeps it with
 *    the identity of the current CUDA context; a call in a later context of that device (after
 *    cudaDeviceReset) looks it up again.  Make the first call on a device, and the first call after a reset,
 *    before any stream capture. */
size_t ms_cvae_static_scratch_bytes(void);
ms_status ms_cvae_train_step_static(const ms_cvae_shape* s, float* params, float* m, float* v, const float* x,
                                    const float* c, const float* eps_z, uint64_t B, uint64_t seed, uint64_t step,
                                    float lr, float weight_decay, float* loss3, void* stream);

/* Walk records -> conditions and targets of the three CVAEs (Sec. 4.1, Eq. 3, Eq. 4 inverted).  Each record
 * is rotated about (0,0,1) by -psi, psi = atan2(x_y, x_x), so the exit point is (sin theta, 0, cos theta);
 * alpha = w~_y, beta = w~_x cos theta - w~_z sin theta.  N is dequantised as y = ln(N - 1/2 + u) with u the
 * 24-bit uniform of word 0 at counter (0, id_lo, id_hi, 0x44), id = photon index.  Outputs (device):
 * cL [n][2] = (ln tau, g), xL [n][1] = y, cP [n][3] = (ln tau, g, ln N), xP [n][3] = (cos theta, alpha,
 * beta), cE [n][7] = (ln tau, g, phi, cos theta, alpha, beta, ln N), xE [n][6] = (X~, W~). */
ms_status ms_training_records(uint64_t n, const int32_t* n_events, const float* exit_pos, const float* exit_dir,
                              const float* rep_pos, const float* rep_dir, const ms_medium* media,
                              int32_t per_photon_media, uint64_t seed, float* cL, float* xL, float* cP,
                              float* xP, float* cE, float* xE, void* stream);

/* ------------------------------------------------------------------------------------------------------
 * Rendering a homogeneous translucent SDF object with a point light (Sec. 3, Fig. 2b; Sec. 4.1; Sec. 4.3,
 * Eq. 5).  The object is the displaced unit sphere f(p) = |p| - 1 - A sin(k x) sin(k y) sin(k z) (negative
 * inside); |f| / (1 + A k) is a conservative distance.  Rays are sphere traced with the largest of that step,
 * the first root of |p + s w| = R(p) +/- A k s (the radial term followed exactly, the displacement bounded;
 * it also detects when the surface is out of reach) and the first root of the curvature bound
 * h + h' s - H s^2 / 2 on the side's distance h (H = A k^2, plus 2 / |p| inside), which closes in on the
 * surface quadratically and steps off it in one step.  The boundary is index matched (no refraction, as in
 * the paper's unrefracted NEE).  Camera paths enter the object; after each free flight to a collision:
 *   MS_SPHERE: if sigma_t * r >= min_optical_radius with r = min(distance bound, max_optical_radius /
 *     sigma_t), one sphere step: LengthGen -> N, PathGen -> exit (Eq. 4), EventGen -> (X, W), NEE at X with
 *     weight Lambda = sum_{i=1..N} phi^i, then absorption with probability 1 - phi^N; otherwise, and always
 *   MS_BRUTE: one scattering event: NEE with weight phi, roulette, HG scattering.
 * The background is black and the light is not visible, so every contribution is a next-event estimate
 * phi-or-Lambda * rho_g(W . w_L) * exp(-sigma_t d_in) * I / |x_L - X|^2.
 * ---------------------------------------------------------------------------------------------------- */
typedef struct {
    int32_t width, height;
    uint32_t spp;               /* samples per pixel; sample indices sample_offset .. +spp-1             */
    uint32_t max_segments;      /* flights per path before truncation                                  */
    float cam_pos[3], cam_at[3], fov_y_deg;
    float light_pos[3], light_I;
    float sigma_t, g, albedo;
    float disp_amp, disp_freq;  /* A, k of the SDF                                                     */
    int32_t mode;               /* MS_BRUTE or MS_SPHERE                                               */
    float min_optical_radius;   /* smallest sigma_t * r for a sphere step (thin-region fallback); <= 0
                                   takes ms_render_default_min_optical_radius(sigma_t)                  */
    float max_optical_radius;   /* largest sigma_t * r (the training range of the models)             */
    uint64_t seed, sample_offset;
    int32_t variant;            /* kernel variant (scheduling constants), 0..ms_render_variants()-1, 0 by
                                   default; in a batch the first request's variant is used           */
    int32_t sdf_grid_n;         /* 0, or the n of sdf_grid                                              */
    const float* sdf_grid;      /* NULL, or device [n][n][n] from ms_sdf_grid_build(disp_amp, disp_freq, n):
                                   a sphere step's radius is then the larger of the distance bound and
                                   the value of the grid voxel holding the collision point             */
    int32_t exact_n1;           /* 0: LengthGen gives N (the paper's form).  1: a sphere step takes N = 1 with
                                   its exact probability exp(-tau) — the first free path from the centre
                                   leaves the sphere (Sec. 3.1) — using the uniform of the tag 4 words'
                                   low bytes, and such a step is exact as a whole: the path leaves
                                   radially along the centre event's HG scattering of the incoming
                                   direction (cos theta from the tag 6 words' low bytes, alpha = beta = 0)
                                   and that event is the representative one.  Otherwise the models give
                                   the step, with N >= 2; for models trained on the N >= 2 records       */
    int32_t phase_timers;       /* 0 normally.  1 (first request of a launch): run an instrumented kernel
                                   of the default variant that also counts shadow-ray march steps in
                                   stats[11] and adds each warp's clock cycles by round kind to the first
                                   request's stats[12..15] (march, decoder, transition, refill) — a time
                                   breakdown; FP32 decoders only; slightly slower                       */
    int32_t exact_centre;       /* 0: EventGen gives the representative event (the paper's form).  1: the
                                   representative event is the step's first event — at the centre, with
                                   the incoming direction — with its exact probability phi / Lambda (the
                                   weight phi^k / Lambda of k = 1, Sec. 4.3; always when N = 1), using the
                                   uniform of the tag 5 words' low bytes, and EventGen, trained on the
                                   records whose representative event is a later one, gives it otherwise;
                                   for models trained that way                                          */
} ms_render_params;

/* The voxel grid of conservative distances that sizes sphere steps (Sec. 3: the bounding volume is voxelised
 * in a pre-process, each voxel holding a conservative shortest distance to the surface).  grid: device
 * [n][n][n] floats, index (iz * n + iy) * n + ix; with h = 2 (1 + disp_amp) / (n - 2) and b = 1 + disp_amp + h,
 * voxel (ix, iy, iz) is the cube [-b + ix h, -b + (ix + 1) h] x ... (one voxel of margin around the bounding
 * sphere).  A voxel may hold surface if |f(c)| <= (1 + A k) h sqrt(3) / 2 at its centre c.  Every voxel's
 * value is (e - sqrt(3)) h, clamped at 0, with e the exact Euclidean distance, in voxels, from its centre to
 * the nearest such voxel's centre (three separable integer passes): two points of two voxels are at most one
 * voxel diagonal, sqrt(3) h, nearer than their centres, so the value is a lower bound of the distance from
 * each of the voxel's points to the surface.  (The paper stores a Chebyshev distance, which is also
 * conservative but up to sqrt(3) smaller along diagonals.)  workspace: device, 16-byte aligned,
 * ms_sdf_grid_workspace_size(n) bytes (two integer grids).  n in 4..1024, 0 <= disp_amp < 1.  Asynchronous on
 * `stream` (five kernel launches: marking, three distance passes, values). */
size_t ms_sdf_grid_workspace_size(int32_t n);
ms_status ms_sdf_grid_build(float disp_amp, float disp_freq, int32_t n, float* grid, void* workspace,
                            size_t workspace_bytes, void* stream);

/* The renderer's three decoders have the final shapes of Table 1 (the paper's D = 2 hidden layers):
 * LengthGen latent 2 width 8, PathGen latent 5 width 16, EventGen latent 5 width 16, all MS_FP32.  A sphere
 * step draws 22 normals n[0..21] (tags 2..7 of its segment, four per tag by Box-Muller): LengthGen z = n[0,1],
 * eps = n[2]; PathGen z = n[3..7], eps = n[8..10]; EventGen z = n[11..15], eps = n[16..21].  Its absorption
 * test and rotation angle psi take the uniforms ((w0 & 0xff) << 16 | (w1 & 0xff) << 8 | (w2 & 0xff)) 2^-24 of
 * the tag 2 and tag 3 words (the low bytes, unused by the normals). */
typedef struct {
    ms_decoder length;          /* LengthGen: p_in 2 (ln tau, g), p_out 1 (ln N dequantised)             */
    ms_decoder path;            /* PathGen:   p_in 3 (ln tau, g, ln N), p_out 3 (cos theta, alpha, beta) */
    ms_decoder event;           /* EventGen:  p_in 7 (ln tau, g, phi, cos theta, alpha, beta, ln N),
                                   p_out 6 (X~, W~)                                                      */
} ms_cvae_set;

size_t ms_render_workspace_size(const ms_render_params* reqs, int n_requests);

/* The thin-region fallback policy (Sec. 6): the minimum optical radius sigma_t r of a sphere step that a request
 * with min_optical_radius <= 0 uses at density sigma_t.  Chosen per density as the threshold of lowest
 * time x squared error against a brute-force reference (the displaced-sphere scene, the trained decoders),
 * interpolated in log sigma_t between the measured densities and held constant beyond them.  Host only. */
float ms_render_default_min_optical_radius(float sigma_t);

/* image: device [height][width] doubles, accumulated: the sum over the pixel's samples (divide by spp).
 * stats: device [MS_RENDER_STATS] accumulated: [0] camera paths, [1] paths entering the object, [2] flights,
 * [3] sphere steps, [4] brute-force events, [5] absorbed, [6] truncated paths or dropped estimates,
 * [7] next-event estimates, [8] SDF evaluations (march steps, each with f's derivative along the ray, and
 * sphere radii at collisions), [9] march steps in the boundary band, [10] completion time
 * of the request in ns after the launch's first block started (written, not accumulated), [11..15] zero
 * (with phase_timers: [11] shadow-ray march steps, [12..15] of the first request the warps' cycles in march,
 * decoder, transition and refill rounds).
 * models: host struct with device weight pointers (ignored in MS_BRUTE).  workspace:
 * ms_render_workspace_size() bytes (sample ticket, start time, finished-path counters).  One persistent
 * launch; asynchronous; capturable in a CUDA graph (a memset and a kernel). */
#define MS_RENDER_STATS 16
ms_status ms_render(const ms_render_params* p, const ms_cvae_set* models, double* image,
                    unsigned long long* stats, void* workspace, size_t workspace_bytes, void* stream);

/* Many requests (1..64) in one persistent launch.  reqs: host [n]; images: device, request i's [h][w] image
 * starts at the sum of the previous requests' h*w; stats: device [n][MS_RENDER_STATS]. */
ms_status ms_render_batch(const ms_render_params* reqs, int n, const ms_cvae_set* models, double* images,
                          unsigned long long* stats, void* workspace, size_t workspace_bytes, void* stream);

/* Kernel variants of the renderer and a native autotuner.  A variant fixes the renderer's scheduling
 * constants (how many parked lanes trigger a decoder round, how many finished marches trigger a transition
 * round, signed-distance steps between scheduling decisions, resident blocks per SM).  ms_render_autotune
 * renders `reqs` (a representative, usually reduced, set of requests) `repeats` times with every variant,
 * timed with CUDA events on `stream`, and returns the fastest in *best_variant (and each variant's time in
 * ms_per_variant[ms_render_variants()] if not NULL).  It waits for the stream; `images` and `stats` are used
 * as scratch (they hold accumulated results of all the runs afterwards). */
int ms_render_variants(void);
ms_status ms_render_variant_info(int i, int* decode_batch, int* trans_batch, int* steps, int* min_blocks);
ms_status ms_render_autotune(const ms_render_params* reqs, int n, const ms_cvae_set* models, double* images,
                             unsigned long long* stats, void* workspace, size_t workspace_bytes, int repeats,
                             int* best_variant, float* ms_per_variant, void* stream);

/* ------------------------------------------------------------------------------------------------------
 * Measured peak issue rates of the execution units that bound the library's ALU-bound kernels: the
 * denominators of the roofline fractions the benchmark reports.  The paper has no counterpart; this is a
 * measurement helper.  ops_per_s: host [MS_PEAK_COUNT], whole-GPU operations (instructions per thread, one
 * per lane) per second: FP32 fused multiply-add (2 flops each), the special-function unit's 2^x, log2 x,
 * sin x and 1/sqrt x approximations, integer multiply-add, three-input logic and high-half multiply.  Each is
 * timed with CUDA events on `stream` in a full-occupancy grid of independent dependency chains; the call waits
 * for the stream.  scratch: device, ms_alu_peaks_scratch_bytes() bytes (each thread's result, so that nothing
 * is optimised away).
 * ---------------------------------------------------------------------------------------------------- */
enum { MS_PEAK_FFMA = 0, MS_PEAK_EX2, MS_PEAK_LG2, MS_PEAK_SIN, MS_PEAK_RSQRT, MS_PEAK_IMAD, MS_PEAK_LOP3,
       MS_PEAK_IMULHI, MS_PEAK_COUNT };
size_t ms_alu_peaks_scratch_bytes(void);
ms_status ms_alu_peaks(double* ops_per_s, void* scratch, size_t scratch_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MS_H */
