/*
 * Oracle: renderer of a homogeneous translucent SDF object — TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain FP64 restatement, one path at a time, of:
 *   Sec. 3 (first paragraph) / Fig. 2b: after a free flight to a collision, take the largest sphere inside
 *       the boundary (from a signed distance function) and bypass the scattering inside it with the learned
 *       models; otherwise (thin region) do one brute-force scattering event.  Delta tracking in a
 *       homogeneous medium is exponential free flight.
 *   Eq. 3: LengthGen samples N (phi = 1 physics), absorption A ~ Bernoulli(1 - phi^N), PathGen samples
 *       (cos theta, alpha, beta), EventGen samples the representative event (X, W).
 *   Eq. 4 and Sec. 4.1: x = r R^CVAE R_psi (sin theta, 0, cos theta); exit direction from (alpha, beta) in
 *       the frame e_n = x^, e_b = w_in x x^, e_t = e_b x e_n; X and W rotated and scaled the same way;
 *       sigma_t -> sigma_t * r before the models are evaluated.
 *   Eq. 5 and Sec. 4.3: next-event estimation toward a point light with transmittance
 *       exp(-sigma_t d_t) along the unrefracted segment; brute force adds phi * rho_g * gamma at every
 *       event, sphere tracing adds Lambda^(N) * rho_g * gamma at the representative event.
 * The readings taken where the paper is silent are listed beside each step below.
 *
 * Mode 2 (exact sampler) runs the same sphere step with the three learned samplers replaced by what they
 * approximate: one brute-force walk in the unit sphere at optical radius sigma_t r (walk.c, the albedo-1
 * physics with the representative event chosen with weights phi^k, i.e. a training record), turned into the
 * models' outputs (N; cos theta, alpha, beta; X~, W~ in the frame where the exit is (sin theta, 0, cos theta))
 * and then put through the same Eq. 4 frame, Lambda, NEE and absorption code as the learned samplers' outputs.
 * Its image must equal the brute-force image in expectation, which pins that composition to the paper's
 * physics.  march_mode 1 replaces the march's step by the plain Lipschitz step |f| / (1 + A k) (Hart's sphere
 * tracing with nothing else), to show that the larger conservative steps find the same crossings.
 *
 * Per path (pixel index -> counter id_hi, sample index -> id_lo) and segment step s (counter word 0):
 *   tag 0: u0 free path, u1 HG cosine, u2 HG azimuth, u3 roulette
 *   tags 2..7: Box-Muller normals n[0..23], tag t words (w0,w1) -> n[4(t-2)], n[4(t-2)+1], (w2,w3) -> next two;
 *       used in order: LengthGen z then eps, PathGen z then eps, EventGen z then eps; the low bytes of words
 *       0..2, which the uniforms leave unused, give ((w0 & 0xff) << 16 | (w1 & 0xff) << 8 | (w2 & 0xff)) 2^-24:
 *       from tag 2 the absorption test's uniform, from tag 3 the rotation angle psi's, from tag 4 the
 *       exact N = 1 test's (exact_n1), from tag 5 the centre-event test's (exact_centre), from tag 6 the
 *       HG cosine of an exact N = 1 step's exit (exact_n1)
 *   tag 8 at step 0: pixel jitter.
 * Uniforms are (w >> 8) * 2^-24 (24-bit), identical to the single-precision kernels' stream.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define R_EPS        1e-4      /* distance from the boundary treated as on it */
#define R_MAX_MARCH  1024      /* sphere-tracing steps per march; a march that runs out ends the path */
#define R_N_MAX      16777216.0
#define R_TAU_CUT    30.0      /* a shadow ray stops once its optical depth inside the medium exceeds this */

typedef struct {
    int32_t p_in, latent, width, p_out;
    const double* w;           /* W1[width][p_in+latent], b1, W2[width][width], b2, W3[2p_out][width], b3 */
} om_decoder;

typedef struct {
    int32_t width, height;
    uint32_t spp, max_segments;
    double cam_pos[3], cam_at[3], fov_y_deg;
    double light_pos[3], light_I;
    double sigma_t, g, albedo;
    double disp_amp, disp_freq;
    int32_t mode;              /* 0 brute force, 1 sphere tracing, 2 sphere tracing with the exact sampler */
    int32_t sdf_grid_n;        /* 0, or n: sphere radii also from an n^3 voxel grid of conservative distances */
    int32_t march_mode;        /* 0 the largest of the three conservative steps, 1 the Lipschitz step alone */
    int32_t max_march;         /* steps per march, 0 for the default R_MAX_MARCH */
    int32_t exact_n1;          /* 1: the N = 1 step drawn exactly (probability exp(-tau), exit along the first
                                  event's HG direction, event at the centre), the models give N >= 2 */
    int32_t exact_centre;      /* 1: the representative event is the first one (the centre, incoming direction)
                                  with its exact probability phi / Lambda, EventGen gives the later ones */
    double min_optical_radius, max_optical_radius;
    uint64_t seed, sample_offset;
    const double* sdf_grid;    /* sdf_grid_n^3 voxel values (index (iz n + iy) n + ix) over [-b, b]^3, voxel side
                                  h = 2 (1 + A) / (n - 2), b = 1 + A + h; each a lower bound of the distance from
                                  the voxel's points to the surface (built by the Python side of the oracle) */
} om_render_params;

typedef struct {
    const om_render_params* P;
    const om_decoder* dec;     /* [3]: LengthGen, PathGen, EventGen (NULL in brute force) */
    const double* grid;        /* the voxel grid (sdf_grid_n > 0), else NULL */
    double* image;
    uint64_t* stats;
    int next_row;
    pthread_mutex_t lock;
} render_job;

static ov3 v3(double x, double y, double z) { ov3 r = { x, y, z }; return r; }
static ov3 add(ov3 a, ov3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static ov3 sub(ov3 a, ov3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static ov3 mul(ov3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
static double dot(ov3 a, ov3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static ov3 cross(ov3 a, ov3 b) { return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static ov3 normalize(ov3 a) { return mul(a, 1.0 / sqrt(dot(a, a))); }

/* ---- scene: displaced unit sphere f(p) = |p| - 1 - A sin(kx) sin(ky) sin(kz), negative inside ---- */
typedef struct {
    double A, k, lip, rb2;
    const double* grid;        /* voxel grid of conservative distances (NULL: none), n^3, index (iz n + iy) n + ix */
    int gn;
    double gb, gh;             /* the grid covers [-gb, gb]^3 in voxels of side gh */
    int plain;                 /* 1: Lipschitz steps only */
    int max_march;             /* steps per march */
} scene;

/* Test hook: a deliberate mistake in the sphere step, so that a test can show its pin catches it (0: none;
 * 1: Lambda summed over i = 0..N; 2: the exit frame's e_t negated; 3: no NEE on a step that absorbs; 4: the
 * representative event not scaled by the sphere's radius). */
static int g_plant = 0;
void om_set_plant(int k) { g_plant = k; }

static _Thread_local uint64_t t_sdf_evals, t_grad_evals;

static double sdf(const scene* S, ov3 p)
{
    t_sdf_evals += 1;
    return sqrt(dot(p, p)) - 1.0 - S->A * sin(S->k * p.x) * sin(S->k * p.y) * sin(S->k * p.z);
}

static ov3 sdf_grad(const scene* S, ov3 p)
{
    double sx = sin(S->k * p.x), sy = sin(S->k * p.y), sz = sin(S->k * p.z);
    double cx = cos(S->k * p.x), cy = cos(S->k * p.y), cz = cos(S->k * p.z);
    double n = sqrt(dot(p, p));
    double ak = S->A * S->k;
    return v3(p.x / n - ak * cx * sy * sz, p.y / n - ak * sx * cy * sz, p.z / n - ak * sx * sy * cz);
}

/*
 * Ray queries of the synthetic scene (the paper traces rays against meshes; this scene is an SDF, and the
 * march is sphere tracing, Hart 1996, with a step bound taken from the form of f).
 * Along p + s w, write f = |p + s w| - R(p + s w) with R(q) = 1 + A sin(kx) sin(ky) sin(kz).  The gradient
 * of sin(kx) sin(ky) sin(kz) has length at most k, so R changes by at most lam s with lam = A k, while the
 * radial term |p + s w| is known exactly along the ray.  Hence, with R0 = R(p) = |p| - f(p):
 *   outside (f > 0):  f(p + s w) >= |p + s w| - R0 - lam s, positive until |p + s w| = R0 + lam s;
 *   inside  (f < 0):  f(p + s w) <= |p + s w| - R0 + lam s, negative until |p + s w| = R0 - lam s.
 * Squaring either equation gives a s^2 + 2 B s + c = 0 with a = 1 - lam^2, c = |p|^2 - R0^2 = f (|p| + R0)
 * and B = p.w -/+ R0 lam; the step is its first positive root, in whichever of the two algebraically equal
 * forms has no cancellation for the sign of B.  Inside there is always exactly one positive root (B < 0 can
 * only happen with lam < 1).  Outside, no positive root (no real root, or B >= 0 with lam <= 1) means the
 * surface cannot be reached along the ray at all: the step is then INFINITY.
 * Every such step is at least the Lipschitz step |f| / (1 + lam), and the callers take the larger of the two.
 */
static double safe_step(const scene* S, ov3 p, ov3 w, double f)
{
    double rp = sqrt(dot(p, p));
    double lam = S->A * S->k;
    double R0 = rp - f;
    double a = 1.0 - lam * lam;
    double c = f * (rp + R0);
    if (f < 0.0) {
        double B = dot(p, w) + R0 * lam;
        double sq = sqrt(fmax(B * B - a * c, 0.0));
        return B >= 0.0 ? -c / (B + sq) : (sq - B) / a;
    }
    double B = dot(p, w) - R0 * lam;
    double disc = B * B - a * c;
    if (disc < 0.0 || (B >= 0.0 && a >= 0.0))
        return INFINITY;
    double sq = sqrt(disc);
    return B < 0.0 ? c / (sq - B) : (B + sq) / -a;
}

/*
 * A second conservative step, from the curvature of f along the ray.  Let h be the marched side's distance
 * function along the ray (h = -f inside the medium, f outside), h0 = h(r) >= 0 and h1 = dh/ds its rate (from
 * the gradient).  Along p + s w, the product sin(kx) sin(ky) sin(kz) is, by
 * sin a sin b sin c = [sin(a+b-c) + sin(a-b+c) + sin(-a+b+c) - sin(a+b+c)] / 4, a sum of four sinusoids of
 * angular frequencies k (+-w1 +-w2 +-w3), so its second derivative in s is at most k^2 / 4 times the sum of the
 * four squared frequencies, i.e. k^2 |w|^2 = k^2; that of |p + s w| lies in [0, 1 / |p + s w|].  So outside
 * h'' >= -H with H = A k^2, and inside, for s <= |r| / 2 (where |p + s w| >= |r| / 2), h'' >= -H with
 * H = A k^2 + 2 / |r|.  Hence h(s) >= h0 + h1 s - H s^2 / 2, which stays positive up to its first positive
 * root (h1 + sqrt(h1^2 + 2 H h0)) / H, written 2 h0 / (sqrt(h1^2 + 2 H h0) - h1) when h1 < 0 (no
 * cancellation): the ray cannot meet the surface before it.  The step is that root, capped at |r| / 2 inside
 * and at 4 outside (past the bounding sphere).  Toward the surface it approaches the crossing quadratically
 * (where the Lipschitz step only closes a fixed fraction of the gap per step); away from it, it leaves the
 * boundary band in one step where steps of the band width would need about lip / h1 of them.
 */
static double curve_step(const scene* S, double rp, double h0, double h1, int inside)
{
    double H = S->A * S->k * S->k + (inside ? 2.0 / rp : 0.0);
    double cap = inside ? 0.5 * rp : 4.0;
    double q = sqrt(h1 * h1 + 2.0 * H * h0);
    double s = h1 < 0.0 ? 2.0 * h0 / (q - h1) : (H > 0.0 ? (h1 + q) / H : cap);
    return fmin(s, cap);
}

/*
 * One march step at r along w on the marched side (inside: the medium).  In the boundary band
 * (|f| / lip < R_EPS) the point counts as on the surface: the ray crosses there when it moves to the other
 * side (*crossing = 1, no step), and otherwise steps off with the curvature step from h0 = max(h, 0), at
 * least R_EPS.  Elsewhere the step is the largest of the three conservative steps (Lipschitz, radial plus
 * Lipschitz, curvature); *escape = 1 when, outside, the surface cannot be reached along the ray.
 */
static double march_step(const scene* S, ov3 r, ov3 w, int inside, int* crossing, int* escape)
{
    double f = sdf(S, r);
    double gd = dot(sdf_grad(S, r), w);
    double h = inside ? -f : f, h1 = inside ? -gd : gd;
    double rp = sqrt(dot(r, r));
    *crossing = 0;
    *escape = 0;
    if (h / S->lip < R_EPS) {
        t_grad_evals += 1;
        if (h1 < 0.0) {
            *crossing = 1;
            return 0.0;
        }
        if (S->plain)
            return R_EPS;
        return fmax(R_EPS, curve_step(S, rp, fmax(h, 0.0), h1, inside));
    }
    if (S->plain)
        return h / S->lip;
    double q = safe_step(S, r, w, f);
    if (q == INFINITY) {
        *escape = 1;
        return INFINITY;
    }
    return fmax(fmax(h / S->lip, q), curve_step(S, rp, h, h1, inside));
}

/* March inside the medium from p along w for at most l.  Returns 1 on a collision (*q = p + l w), 0 when
 * the boundary is crossed outward at *q, 2 when the step cap runs out. */
static int march_inside(const scene* S, ov3 p, ov3 w, double l, ov3* q)
{
    double t = 0.0;
    for (int it = 0; it < S->max_march; ++it) {
        ov3 r = add(p, mul(w, t));
        int crossing, escape;
        double d = march_step(S, r, w, 1, &crossing, &escape);
        if (crossing) {
            *q = r;
            return 0;
        }
        if (t + d >= l) {
            *q = add(p, mul(w, l));
            return 1;
        }
        t = t + d;
    }
    return 2;
}

/* March outside from p along w.  Returns 1 when the path re-enters at *q, 0 when it leaves the bounding
 * sphere, 2 when the step cap runs out. */
static int march_outside(const scene* S, ov3 p, ov3 w, ov3* q)
{
    double t = 0.0;
    for (int it = 0; it < S->max_march; ++it) {
        ov3 r = add(p, mul(w, t));
        if (dot(r, r) > S->rb2 && dot(r, w) >= 0.0)
            return 0;
        int crossing, escape;
        double d = march_step(S, r, w, 0, &crossing, &escape);
        if (crossing) {
            *q = r;
            return 1;
        }
        if (escape)
            return 0;
        t = t + d;
    }
    return 2;
}

/* Length of the straight segment X -> x_L that lies inside the medium (Sec. 4.3, d_t); -1 when the step
 * cap runs out (the estimate is then dropped).  A boundary crossing switches the side at the same point.  The
 * march stops once the inside length exceeds din_cut (returning it): the transmittance exp(-sigma_t d_t) is
 * then below exp(-sigma_t din_cut), and whatever follows can only make it smaller. */
static double inside_length(const scene* S, ov3 X, ov3 xl, double din_cut)
{
    ov3 dl = sub(xl, X);
    double D = sqrt(dot(dl, dl));
    ov3 w = mul(dl, 1.0 / D);
    double t = 0.0, din = 0.0;
    int inside = 1;
    for (int it = 0; it < S->max_march; ++it) {
        if (t >= D || din > din_cut)
            return din;
        ov3 r = add(X, mul(w, t));
        if (!inside && dot(r, r) > S->rb2 && dot(r, w) >= 0.0)
            return din;
        int crossing, escape;
        double d = march_step(S, r, w, inside, &crossing, &escape);
        if (crossing) {
            inside = !inside;
            continue;
        }
        if (escape)
            return din;
        double step = fmin(d, D - t);
        if (inside)
            din = din + step;
        t = t + step;
    }
    return -1.0;
}

/* ---- random numbers ---- */
typedef struct { uint32_t key[2]; uint64_t id; } stream;

static void words(const stream* s, uint32_t step, uint32_t tag, uint32_t w[4])
{
    uint32_t ctr[4] = { step, (uint32_t)s->id, (uint32_t)(s->id >> 32), tag };
    om_philox(ctr, s->key, w);
}
static double u24(uint32_t w) { return (double)(w >> 8) * 0x1.0p-24; }

static void normals(const stream* s, uint32_t step, double n[24], double extra[5])
{
    for (uint32_t t = 2; t < 8; ++t) {
        uint32_t w[4];
        words(s, step, t, w);
        if (t < 7)
            extra[t - 2] = (double)(((w[0] & 0xffu) << 16) | ((w[1] & 0xffu) << 8) | (w[2] & 0xffu)) * 0x1.0p-24;
        for (int pair = 0; pair < 2; ++pair) {
            double ua = u24(w[2 * pair]), ub = u24(w[2 * pair + 1]);
            double r = sqrt(-2.0 * log(1.0 - ua));
            n[4 * (t - 2) + 2 * pair] = r * cos(2.0 * M_PI * ub);
            n[4 * (t - 2) + 2 * pair + 1] = r * sin(2.0 * M_PI * ub);
        }
    }
}

/* ---- learned models (Sec. 3.2): decoder MLP with Softplus between hidden layers ---- */
static double softplus(double x) { return fmax(x, 0.0) + log1p(exp(-fabs(x))); }

static void decoder_eval(const om_decoder* D, const double* in, double* out)
{
    int nin = D->p_in + D->latent, W = D->width, no = 2 * D->p_out;
    const double* W1 = D->w;
    const double* b1 = W1 + W * nin;
    const double* W2 = b1 + W;
    const double* b2 = W2 + W * W;
    const double* W3 = b2 + W;
    const double* b3 = W3 + no * W;
    double h1[64], h2[64];
    for (int i = 0; i < W; ++i) {
        double a = b1[i];
        for (int j = 0; j < nin; ++j) a += W1[i * nin + j] * in[j];
        h1[i] = softplus(a);
    }
    for (int i = 0; i < W; ++i) {
        double a = b2[i];
        for (int j = 0; j < W; ++j) a += W2[i * W + j] * h1[j];
        h2[i] = softplus(a);
    }
    for (int i = 0; i < no; ++i) {
        double a = b3[i];
        for (int j = 0; j < W; ++j) a += W3[i * W + j] * h2[j];
        out[i] = a;
    }
}

/* Draw one decoder sample x = mu + sqrt(Sigma) * eps (Sec. 3.2) from condition c and normals z, eps. */
static void decoder_sample(const om_decoder* D, const double* c, const double* z, const double* eps, double* x)
{
    double in[32], out[32];
    for (int j = 0; j < D->p_in; ++j) in[j] = c[j];
    for (int j = 0; j < D->latent; ++j) in[D->p_in + j] = z[j];
    decoder_eval(D, in, out);
    for (int j = 0; j < D->p_out; ++j)
        x[j] = out[j] + exp(0.5 * out[D->p_out + j]) * eps[j];
}

/* ---- phase function (Eq. 1) and its sampling ---- */
static double hg_pdf(double cosang, double g)
{
    double den = 1.0 + g * g - 2.0 * g * cosang;
    return (1.0 - g * g) / (4.0 * M_PI * den * sqrt(den));
}

static double hg_cosine(double u, double g)
{
    if (fabs(g) < 1e-4)
        return 2.0 * u - 1.0;
    double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
    return fmin(1.0, fmax(-1.0, (1.0 + g * g - t * t) / (2.0 * g)));
}

/* Orthonormal basis (t1, t2, w) of Duff et al. 2017; R^CVAE maps (0,0,1) to w. */
static void onb(ov3 w, ov3* t1, ov3* t2)
{
    double sign = w.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sign + w.z);
    double b = w.x * w.y * a;
    *t1 = v3(1.0 + sign * w.x * w.x * a, sign * b, -sign * w.x);
    *t2 = v3(b, sign + w.y * w.y * a, -w.y);
}

static ov3 scatter_dir(ov3 w, double mu, double u)
{
    ov3 t1, t2;
    onb(w, &t1, &t2);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double ph = 2.0 * M_PI * u;
    return normalize(add(add(mul(t1, st * cos(ph)), mul(t2, st * sin(ph))), mul(w, mu)));
}

/* Next-event estimate toward the point light from X, arriving with direction W (Eq. 5 term). */
/* The grid value of the voxel holding p (the voxel index clamped to the grid). */
static double grid_value(const scene* S, ov3 p)
{
    int i[3];
    double c[3] = { p.x, p.y, p.z };
    for (int a = 0; a < 3; ++a) {
        int v = (int)floor((c[a] + S->gb) / S->gh);
        i[a] = v < 0 ? 0 : (v > S->gn - 1 ? S->gn - 1 : v);
    }
    return S->grid[((size_t)i[2] * S->gn + i[1]) * S->gn + i[0]];
}

static double nee(const scene* S, const om_render_params* P, ov3 X, ov3 W, double weight, uint64_t* st)
{
    ov3 xl = v3(P->light_pos[0], P->light_pos[1], P->light_pos[2]);
    ov3 dl = sub(xl, X);
    double d2 = dot(dl, dl);
    ov3 wl = mul(dl, 1.0 / sqrt(d2));
    double rho = hg_pdf(dot(W, wl), P->g);
    /* a shadow ray whose optical depth passes R_TAU_CUT is not marched further: its transmittance is below
     * exp(-R_TAU_CUT) (about 1e-13) of the unshadowed term, far below single precision and Monte Carlo noise */
    double din = inside_length(S, X, xl, R_TAU_CUT / P->sigma_t);
    if (din < 0.0) {
        st[6] += 1;
        return 0.0;
    }
    return weight * rho * exp(-P->sigma_t * din) * P->light_I / d2;
}

int om_walk_record(uint64_t seed, uint64_t id, double tau, double g, double phi, uint32_t max_events,
                   int32_t* n, double x[3], double w[3], double X[3], double W[3]);

/*
 * The exact sampler of one sphere step: a walk record at optical radius tau (N, exit x and w, representative
 * event X and W, the albedo-1 physics with weights phi^k), drawn on its own stream (key: the render seed mixed
 * with the segment, counter id: the path's), turned into the three models' outputs (Sec. 4.1): rotated about
 * (0,0,1) by -psi_exit, psi_exit = atan2(x_y, x_x), so that the exit is (sin theta, 0, cos theta); then
 * cos theta = x~_z, alpha = w~ . e_b = w~_y, beta = w~ . e_t = w~_x cos theta - w~_z sin theta, and (X~, W~)
 * the rotated event.  Returns 0 when the walk ran out of events.
 */
static int exact_sample(const om_render_params* P, uint64_t id, uint32_t seg, double tau, double* N, double* ct,
                        double* al, double* be, double xe[6])
{
    uint64_t key = P->seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(seg + 1u));
    int32_t n = 0;
    double x[3], w[3], X[3], W[3];
    if (om_walk_record(key, id, tau, P->g, P->albedo, 1u << 24, &n, x, w, X, W) != 0)
        return 0;
    double ps = atan2(x[1], x[0]);
    double c = cos(ps), s = sin(ps);
    double xr[3] = { c * x[0] + s * x[1], -s * x[0] + c * x[1], x[2] };
    double wr[3] = { c * w[0] + s * w[1], -s * w[0] + c * w[1], w[2] };
    *N = (double)n;
    *ct = xr[2];
    *al = wr[1];
    *be = wr[0] * xr[2] - wr[2] * xr[0];
    xe[0] = c * X[0] + s * X[1]; xe[1] = -s * X[0] + c * X[1]; xe[2] = X[2];
    xe[3] = c * W[0] + s * W[1]; xe[4] = -s * W[0] + c * W[1]; xe[5] = W[2];
    return 1;
}

/* One camera path; returns its contribution and updates the counters. */
static double trace_path(const render_job* J, const scene* S, int px, int py, uint64_t sample, uint64_t* st)
{
    const om_render_params* P = J->P;
    stream rs;
    rs.key[0] = (uint32_t)P->seed;
    rs.key[1] = (uint32_t)(P->seed >> 32);
    rs.id = ((uint64_t)(uint32_t)(py * P->width + px) << 32) | (uint32_t)sample;
    uint32_t w4[4];
    words(&rs, 0u, 8u, w4);
    double jx = u24(w4[0]), jy = u24(w4[1]);

    /* pinhole camera */
    ov3 cp = v3(P->cam_pos[0], P->cam_pos[1], P->cam_pos[2]);
    ov3 fw = normalize(sub(v3(P->cam_at[0], P->cam_at[1], P->cam_at[2]), cp));
    ov3 rt = normalize(cross(fw, v3(0.0, 1.0, 0.0)));
    ov3 up = cross(rt, fw);
    double th = tan(0.5 * P->fov_y_deg * M_PI / 180.0);
    double aspect = (double)P->width / (double)P->height;
    double sx = (2.0 * ((double)px + jx) / (double)P->width - 1.0) * th * aspect;
    double sy = (1.0 - 2.0 * ((double)py + jy) / (double)P->height) * th;
    ov3 w = normalize(add(add(fw, mul(rt, sx)), mul(up, sy)));

    st[0] += 1;
    ov3 p;
    int hit = march_outside(S, cp, w, &p);
    if (hit != 1) {
        st[6] += (uint64_t)(hit == 2);
        return 0.0;
    }
    st[1] += 1;

    const double sig = P->sigma_t, g = P->g, phi = P->albedo;
    double acc = 0.0;
    for (uint32_t seg = 0;; ++seg) {
        if (seg >= P->max_segments) {
            st[6] += 1;
            break;
        }
        st[2] += 1;
        uint32_t u[4];
        words(&rs, seg, 0u, u);
        double l = -log(1.0 - u24(u[0])) / sig;
        ov3 c;
        int ev = march_inside(S, p, w, l, &c);
        if (ev == 2) {
            st[6] += 1;
            break;
        }
        if (ev == 0) {
            ov3 re;
            int back = march_outside(S, c, w, &re);
            if (back != 1) {
                st[6] += (uint64_t)(back == 2);
                break;                      /* left the object: black background */
            }
            p = re;                         /* re-entered: fresh flight (memoryless) */
            continue;
        }
        if (P->mode == 1 || P->mode == 2) {
            double d = -sdf(S, c) / S->lip;
            if (S->grid)
                d = fmax(d, grid_value(S, c));
            double r = fmin(d, P->max_optical_radius / sig);
            double tau = sig * r;
            if (tau >= P->min_optical_radius) {
                /* ---- sphere-tracing step: the three models of Eq. 3 at optical radius tau ---- */
                st[3] += 1;
                double n[24], ua[5];
                normals(&rs, seg, n, ua);
                double N, ct, al, be, ab2, xe[6];
                if (P->mode == 2) {
                    if (!exact_sample(P, rs.id, seg, tau, &N, &ct, &al, &be, xe)) {
                        st[6] += 1;
                        break;
                    }
                    ab2 = al * al + be * be;
                } else {
                    /* the normals are used in order: each model's z (its latent size), then its eps (its
                     * output size) — LengthGen, PathGen, EventGen */
                    const om_decoder* D = J->dec;
                    int zL = 0, eL = zL + D[0].latent, zP = eL + D[0].p_out, eP = zP + D[1].latent;
                    int zE = eP + D[1].p_out, eE = zE + D[2].latent;
                    double ltau = log(tau);
                    double cL[2] = { ltau, g }, yN;
                    decoder_sample(&D[0], cL, n + zL, n + eL, &yN);
                    N = floor(exp(yN) + 0.5);
                    /* exact_n1: a step leaves the sphere after its first event (at the centre) exactly when the
                     * first free path exceeds the radius, with probability exp(-tau) (Sec. 3.1); that mass is
                     * drawn as such and LengthGen, trained on the N >= 2 records, gives the rest.  Such a step
                     * is then exact as a whole: the path leaves radially along the event's HG scattering of the
                     * incoming direction, so x~ = w~ = (sin theta, 0, cos theta) with cos theta the HG cosine
                     * and alpha = beta = 0, and its one event, the centre, is the representative one */
                    double n_min = P->exact_n1 ? 2.0 : 1.0;
                    if (!(N >= n_min)) N = n_min;
                    if (N > R_N_MAX) N = R_N_MAX;
                    if (P->exact_n1 && ua[2] < exp(-tau))
                        N = 1.0;
                    double lnN = log(N);
                    double cP[3] = { ltau, g, lnN }, xp[3];
                    decoder_sample(&D[1], cP, n + zP, n + eP, xp);
                    ct = fmin(1.0, fmax(-1.0, xp[0]));
                    al = xp[1];
                    be = xp[2];
                    ab2 = al * al + be * be;
                    if (ab2 > 1.0) {
                        double s = 1.0 / sqrt(ab2);
                        al = al * s; be = be * s; ab2 = 1.0;
                    }
                    double cE[7] = { ltau, g, phi, ct, al, be, lnN };
                    decoder_sample(&D[2], cE, n + zE, n + eE, xe);
                    if (P->exact_n1 && N <= 1.0) {
                        ct = hg_cosine(ua[4], g);
                        al = 0.0; be = 0.0; ab2 = 0.0;
                    }
                }
                double phiN = pow(phi, N);
                double lam = (phi < 1.0) ? phi * (1.0 - phiN) / (1.0 - phi) : N;
                /* exact_centre: the first event sits at the centre c with the incoming direction w, and Sec. 4.3
                 * picks it as the representative event with probability phi / Lambda^(N) (k = 1); that atom,
                 * which a Gaussian decoder cannot form, is drawn as such, and EventGen, trained on the records
                 * whose representative event is a later one, gives the rest */
                int centre = N <= 1.0 ? (P->exact_n1 || P->exact_centre) : (P->exact_centre && ua[3] < phi / lam);
                if (P->mode == 1 && centre) {
                    xe[0] = 0.0; xe[1] = 0.0; xe[2] = 0.0;
                    xe[3] = 0.0; xe[4] = 0.0; xe[5] = 1.0;
                }
                if (g_plant == 1)
                    lam = lam + 1.0;

                /* Eq. 4 and Sec. 4.1: CVAE frame -> world */
                ov3 t1, t2;
                onb(w, &t1, &t2);
                double psi = 2.0 * M_PI * ua[1];
                double cs = cos(psi), sn = sin(psi);
                double stt = sqrt(fmax(0.0, 1.0 - ct * ct));
                double nn = sqrt(fmax(0.0, 1.0 - ab2));
                double bt = g_plant == 2 ? -be : be;
                ov3 xt = v3(stt, 0.0, ct);
                ov3 wt = v3(bt * ct + nn * stt, al, -bt * stt + nn * ct);
                ov3 Xt = v3(xe[0], xe[1], xe[2]);
                double xn = sqrt(dot(Xt, Xt));
                if (xn > 1.0) Xt = mul(Xt, 1.0 / xn);
                ov3 Wt = v3(xe[3], xe[4], xe[5]);
                double wn = sqrt(dot(Wt, Wt));
                Wt = wn > 1e-12 ? mul(Wt, 1.0 / wn) : v3(0.0, 0.0, 1.0);
                ov3 vs[4] = { xt, wt, Xt, Wt }, vw[4];
                for (int k = 0; k < 4; ++k) {
                    ov3 v1 = v3(cs * vs[k].x - sn * vs[k].y, sn * vs[k].x + cs * vs[k].y, vs[k].z);
                    vw[k] = add(add(mul(t1, v1.x), mul(t2, v1.y)), mul(w, v1.z));
                }
                ov3 xexit = add(c, mul(vw[0], r));
                ov3 wout = normalize(vw[1]);
                ov3 X = add(c, mul(vw[2], g_plant == 4 ? 1.0 : r));
                ov3 Wd = normalize(vw[3]);
                st[7] += 1;
                int absorbed = ua[0] >= phiN;
                if (!(g_plant == 3 && absorbed))
                    acc += nee(S, P, X, Wd, lam, st);
                if (absorbed) {
                    st[5] += 1;
                    break;
                }
                p = xexit;
                w = wout;
                continue;
            }
        }
        /* ---- brute-force scattering event (Sec. 3.1) with next-event estimation (Eq. 5) ---- */
        st[4] += 1;
        st[7] += 1;
        acc += nee(S, P, c, w, phi, st);
        if (u24(u[3]) >= phi) {
            st[5] += 1;
            break;
        }
        w = scatter_dir(w, hg_cosine(u24(u[1]), g), u24(u[2]));
        p = c;
    }
    return acc;
}

static void* render_worker(void* arg)
{
    render_job* J = (render_job*)arg;
    const om_render_params* P = J->P;
    scene S;
    S.A = P->disp_amp;
    S.k = P->disp_freq;
    S.lip = 1.0 + P->disp_amp * P->disp_freq;
    double rb = 1.0 + P->disp_amp + 1e-3;
    S.rb2 = rb * rb;
    S.grid = J->grid;
    S.gn = P->sdf_grid_n;
    S.gh = S.grid ? 2.0 * (1.0 + S.A) / (double)(S.gn - 2) : 0.0;
    S.gb = 1.0 + S.A + S.gh;
    S.plain = P->march_mode == 1;
    S.max_march = P->max_march > 0 ? P->max_march : R_MAX_MARCH;
    uint64_t st[16] = { 0 };
    t_sdf_evals = 0;
    t_grad_evals = 0;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int py = J->next_row++;
        pthread_mutex_unlock(&J->lock);
        if (py >= P->height)
            break;
        for (int px = 0; px < P->width; ++px) {
            double acc = 0.0;
            for (uint32_t s = 0; s < P->spp; ++s)
                acc += trace_path(J, &S, px, py, P->sample_offset + s, st);
            J->image[(size_t)py * P->width + px] += acc;
        }
    }
    st[8] = t_sdf_evals;
    st[9] = t_grad_evals;
    pthread_mutex_lock(&J->lock);
    for (int k = 0; k < 16; ++k) J->stats[k] += st[k];
    pthread_mutex_unlock(&J->lock);
    return NULL;
}

/*
 * Render: image[h][w] accumulates the sum over the spp samples of each pixel (divide by spp for the mean).
 * stats[16]: camera paths, paths entering the object, flight segments, sphere steps, brute events,
 * absorbed paths, truncated paths or dropped estimates (segment cap or march step cap), next-event
 * estimates, SDF evaluations (distance and gradient), boundary-band steps, zeros.  Returns the number of threads used.
 */
int om_render(const om_render_params* P, const om_decoder* dec3, double* image, uint64_t* stats, int n_threads)
{
    if (P->mode == 1 && dec3) {
        int used = 0;
        for (int k = 0; k < 3; ++k) {
            if (dec3[k].width > 64 || dec3[k].p_in + dec3[k].latent > 64) return -1;
            used += dec3[k].latent + dec3[k].p_out;
        }
        if (used > 24) return -1;   /* a sphere step draws 24 normals */
    }
    const double* grid = NULL;
    if (P->mode != 0 && P->sdf_grid_n > 0) {
        if (P->sdf_grid_n < 4 || P->disp_amp >= 1.0 || !P->sdf_grid) return -1;
        grid = P->sdf_grid;
    }
    render_job J;
    J.P = P;
    J.dec = dec3;
    J.grid = grid;
    J.image = image;
    J.stats = stats;
    J.next_row = 0;
    pthread_mutex_init(&J.lock, NULL);
    int nt = om_num_threads(n_threads);
    if (nt > P->height) nt = P->height > 0 ? P->height : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        pthread_create(&th[t], NULL, render_worker, &J);
    for (int t = 0; t < nt; ++t)
        pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    return nt;
}

/*
 * Selected pixels of the same render: values[i] = the sum over the spp samples of pixel pixels[i] (index
 * py * width + px), on exactly the streams the whole-image render uses for that pixel; stats as om_render.
 * Lets a test check sampled pixels of a full-size render one by one.  Returns the threads used, or -1.
 */
typedef struct {
    render_job* J;
    const int64_t* pixels;
    int n_pixels;
    double* values;
    int next;
} pixel_job;

static void* pixel_worker(void* arg)
{
    pixel_job* Q = (pixel_job*)arg;
    render_job* J = Q->J;
    const om_render_params* P = J->P;
    scene S;
    S.A = P->disp_amp;
    S.k = P->disp_freq;
    S.lip = 1.0 + P->disp_amp * P->disp_freq;
    double rb = 1.0 + P->disp_amp + 1e-3;
    S.rb2 = rb * rb;
    S.grid = J->grid;
    S.gn = P->sdf_grid_n;
    S.gh = S.grid ? 2.0 * (1.0 + S.A) / (double)(S.gn - 2) : 0.0;
    S.gb = 1.0 + S.A + S.gh;
    S.plain = P->march_mode == 1;
    S.max_march = P->max_march > 0 ? P->max_march : R_MAX_MARCH;
    uint64_t st[16] = { 0 };
    t_sdf_evals = 0;
    t_grad_evals = 0;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int i = Q->next++;
        pthread_mutex_unlock(&J->lock);
        if (i >= Q->n_pixels)
            break;
        int px = (int)(Q->pixels[i] % P->width), py = (int)(Q->pixels[i] / P->width);
        double acc = 0.0;
        for (uint32_t smp = 0; smp < P->spp; ++smp)
            acc += trace_path(J, &S, px, py, P->sample_offset + smp, st);
        Q->values[i] = acc;
    }
    st[8] = t_sdf_evals;
    st[9] = t_grad_evals;
    pthread_mutex_lock(&J->lock);
    for (int k = 0; k < 16; ++k) J->stats[k] += st[k];
    pthread_mutex_unlock(&J->lock);
    return NULL;
}

int om_render_pixels(const om_render_params* P, const om_decoder* dec3, const int64_t* pixels, int n_pixels,
                     double* values, uint64_t* stats, int n_threads)
{
    if (n_pixels < 0 || (n_pixels > 0 && (!pixels || !values)))
        return -1;
    for (int i = 0; i < n_pixels; ++i)
        if (pixels[i] < 0 || pixels[i] >= (int64_t)P->width * P->height)
            return -1;
    if (P->mode == 1 && dec3) {
        int used = 0;
        for (int k = 0; k < 3; ++k) {
            if (dec3[k].width > 64 || dec3[k].p_in + dec3[k].latent > 64) return -1;
            used += dec3[k].latent + dec3[k].p_out;
        }
        if (used > 24) return -1;
    }
    const double* grid = NULL;
    if (P->mode != 0 && P->sdf_grid_n > 0) {
        if (P->sdf_grid_n < 4 || P->disp_amp >= 1.0 || !P->sdf_grid) return -1;
        grid = P->sdf_grid;
    }
    render_job J;
    J.P = P;
    J.dec = dec3;
    J.grid = grid;
    J.image = NULL;
    J.stats = stats;
    J.next_row = 0;
    pthread_mutex_init(&J.lock, NULL);
    pixel_job Q = { &J, pixels, n_pixels, values, 0 };
    int nt = om_num_threads(n_threads);
    if (nt > n_pixels) nt = n_pixels > 0 ? n_pixels : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        pthread_create(&th[t], NULL, pixel_worker, &Q);
    for (int t = 0; t < nt; ++t)
        pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    return nt;
}

/* Single-query decoder sample, exposed for the tests. */
void om_decoder_sample(const om_decoder* D, const double* c, const double* z, const double* eps, double* x)
{
    decoder_sample(D, c, z, eps, x);
}

/* First boundary crossing along p + t w, exposed for the tests: from outside (f(p) > 0) the re-entry
 * march, from inside the exit march with no collision, with the three-bound step (plain = 0) or the Lipschitz
 * step alone (plain = 1, with a step cap of 2^22).  Returns 1 with *t at the crossing, 0 when an outside ray
 * escapes, 2 when the step cap runs out. */
int om_ray_crossing(double A, double k, const double* p, const double* w, double* t, int plain)
{
    scene S = { A, k, 1.0 + A * k, (1.0 + A + 1e-3) * (1.0 + A + 1e-3), NULL, 0, 0.0, 0.0, plain != 0,
                plain ? (1 << 22) : R_MAX_MARCH };
    ov3 o = v3(p[0], p[1], p[2]), d = v3(w[0], w[1], w[2]), q = o;
    int r;
    if (sdf(&S, o) > 0.0) {
        r = march_outside(&S, o, d, &q);
    } else {
        r = march_inside(&S, o, d, INFINITY, &q);
        r = r == 0 ? 1 : 2;
    }
    *t = sqrt(dot(sub(q, o), sub(q, o)));
    return r;
}

/* The band step from p along w (the side is that of f(p)); -1 when the ray meets the surface there (it
 * moves toward it), exposed for the tests. */
double om_band_step(double A, double k, const double* p, const double* w)
{
    scene S = { A, k, 1.0 + A * k, (1.0 + A + 1e-3) * (1.0 + A + 1e-3), NULL, 0, 0.0, 0.0, 0, R_MAX_MARCH };
    ov3 r = v3(p[0], p[1], p[2]), d = v3(w[0], w[1], w[2]);
    double f = sdf(&S, r);
    int inside = f < 0.0;
    double gd = dot(sdf_grad(&S, r), d);
    double h = inside ? -f : f, h1 = inside ? -gd : gd;
    return h1 < 0.0 ? -1.0 : fmax(R_EPS, curve_step(&S, sqrt(dot(r, r)), fmax(h, 0.0), h1, inside));
}

/* One march step from p along w on the side of f(p): -1 for a crossing, INFINITY for an escape, exposed
 * for the tests. */
double om_march_step(double A, double k, const double* p, const double* w)
{
    scene S = { A, k, 1.0 + A * k, (1.0 + A + 1e-3) * (1.0 + A + 1e-3), NULL, 0, 0.0, 0.0, 0, R_MAX_MARCH };
    ov3 r = v3(p[0], p[1], p[2]), d = v3(w[0], w[1], w[2]);
    int crossing, escape;
    double s = march_step(&S, r, d, sdf(&S, r) < 0.0, &crossing, &escape);
    return crossing ? -1.0 : s;
}

/* Inside length of one segment, exposed for the tests. */
double om_inside_length(double A, double k, const double* X, const double* xl)
{
    scene S = { A, k, 1.0 + A * k, (1.0 + A + 1e-3) * (1.0 + A + 1e-3), NULL, 0, 0.0, 0.0, 0, R_MAX_MARCH };
    return inside_length(&S, v3(X[0], X[1], X[2]), v3(xl[0], xl[1], xl[2]), INFINITY);
}
