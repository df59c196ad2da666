/*
 * Oracle: brute-force Henyey-Greenstein random walk in the unit sphere — TEST INFRASTRUCTURE ONLY.
 *
 * Sec. 3.1: photons start at the centre of a sphere of unit radius with incoming direction w_in; the first
 * scattering event happens at the centre; free paths are l = -log(1 - xi) / sigma_t; at every event Russian
 * roulette continues the path with probability phi (the albedo), and the new direction is drawn from the
 * HG phase function (Eq. 1), whose mean cosine is g; the walk ends when the path first crosses the sphere.
 * Sec. 4.3: one representative event k is chosen with probability phi^k / Lambda^(N); it is found here
 * with a streaming (one-pass) weighted reservoir over the events.
 *
 * Random numbers per photon id and event step s (counter = (s, id_lo, id_hi, tag), key = seed):
 *   tag 0 words (hi) and, for 53-bit uniforms, tag 2 words (lo):
 *       u0 free path, u1 HG cosine (or start z), u2 azimuth, u3 roulette;
 *       the reservoir uniform from the bits those four leave unused: with 24-bit uniforms
 *       ((hi0 & 0xff) << 16 | (hi1 & 0xff) << 8 | (hi2 & 0xff)) * 2^-24, with 53-bit uniforms
 *       ((lo0 & 0x7ff) << 22 | (lo1 & 0x7ff) << 11 | (lo2 & 0x7ff)) * 2^-33;
 *   tag 1 (hi) / tag 3 (lo): a2 a3 isotropic start direction when an event sits at the centre.
 * A 53-bit uniform is ((hi << 21) | (lo >> 11)) * 2^-53; a 24-bit uniform is (hi >> 8) * 2^-24.
 *
 * Everything is FP64 with only basic operations and the deterministic log/sincos/atan2 of detmath.c, so
 * that an implementation performing the same steps in the same order reproduces every integer exactly.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>
#include "oracle.h"

#define OM_PI   0x1.921fb54442d18p+1
#define OM_2PI  0x1.921fb54442d18p+2

enum { OM_ESCAPED = 0, OM_ABSORBED = 1, OM_TRUNCATED = 2 };

typedef struct {
    uint64_t seed, photon_offset, n_photons;
    const om_medium* media;
    int per_photon_media;
    uint32_t max_events;
    int reservoir_mode;   /* 0 none, 1 uniform over events, 2 weights phi^k with roulette off */
    int uniform_bits;     /* 53 or 24 */
    int32_t* n_events;
    uint8_t* status;
    double *exit_pos, *exit_dir, *rep_pos, *rep_dir;
    int32_t* rep_index;
    uint64_t *hist_n, *hist_pos, *hist_cos, *counters;
    pthread_mutex_t lock;
    const double* nee_light;   /* optional: a point light outside the unit sphere; then nee_sum[i] receives */
    double* nee_sum;           /* sum_k phi^k rho_g(W_k . w_L) exp(-tau d_k) / |x_L - X_k|^2 over the events */
} walk_job;

typedef struct {
    walk_job* job;
    uint64_t begin, end;
} walk_chunk;

int om_num_threads(int requested)
{
    if (requested > 0)
        return requested;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static double dot3(ov3 a, ov3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

static void draw(const walk_job* J, uint64_t id, uint32_t step, uint32_t tag_hi, double u[4], double* ures)
{
    uint32_t key[2] = { (uint32_t)J->seed, (uint32_t)(J->seed >> 32) };
    uint32_t ctr[4] = { step, (uint32_t)id, (uint32_t)(id >> 32), tag_hi };
    uint32_t hi[4];
    om_philox(ctr, key, hi);
    if (J->uniform_bits == 24) {
        for (int j = 0; j < 4; ++j)
            u[j] = (double)(hi[j] >> 8) * 0x1.0p-24;
        if (ures)
            *ures = (double)(((hi[0] & 0xffu) << 16) | ((hi[1] & 0xffu) << 8) | (hi[2] & 0xffu)) * 0x1.0p-24;
        return;
    }
    uint32_t lo[4];
    ctr[3] = tag_hi + 2u;
    om_philox(ctr, key, lo);
    for (int j = 0; j < 4; ++j)
        u[j] = (double)(((uint64_t)hi[j] << 21) | (uint64_t)(lo[j] >> 11)) * 0x1.0p-53;
    if (ures)
        *ures = (double)(((uint64_t)(lo[0] & 0x7ffu) << 22) | ((uint64_t)(lo[1] & 0x7ffu) << 11) |
                         (uint64_t)(lo[2] & 0x7ffu)) * 0x1.0p-33;
}

/* Inverse CDF of the HG phase function (Eq. 1): cosine between old and new propagation direction. */
double om_hg_cosine(double u, double g)
{
    if (fabs(g) < 1e-4)
        return 2.0 * u - 1.0;
    double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
    double mu = (1.0 + g * g - t * t) / (2.0 * g);
    if (mu < -1.0) mu = -1.0;
    if (mu > 1.0) mu = 1.0;
    return mu;
}

/* New direction at polar cosine mu and azimuth 2*pi*u around w, in the branch-free orthonormal basis of
 * Duff et al. (JCGT 2017), renormalised. */
static ov3 scatter_dir(ov3 w, double mu, double u)
{
    double sign = (w.z >= 0.0) ? 1.0 : -1.0;
    double a = -1.0 / (sign + w.z);
    double b = w.x * w.y * a;
    ov3 t1 = { 1.0 + sign * w.x * w.x * a, sign * b, -sign * w.x };
    ov3 t2 = { b, sign + w.y * w.y * a, -w.y };
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double sp, cp;
    om_sincos_turns(u, &sp, &cp);
    double ca = st * cp, sa = st * sp;
    ov3 r = { ca * t1.x + sa * t2.x + mu * w.x,
              ca * t1.y + sa * t2.y + mu * w.y,
              ca * t1.z + sa * t2.z + mu * w.z };
    double n = sqrt(dot3(r, r));
    r.x = r.x / n; r.y = r.y / n; r.z = r.z / n;
    return r;
}

static ov3 iso_dir(double uz, double uphi)
{
    double z = 1.0 - 2.0 * uz;
    double st = sqrt(fmax(0.0, 1.0 - z * z));
    double sp, cp;
    om_sincos_turns(uphi, &sp, &cp);
    ov3 r = { st * cp, st * sp, z };
    return r;
}

/* Test hook: the rotation used at every event. */
void om_scatter_dir(const double* w, double mu, double u, double* out)
{
    ov3 a = { w[0], w[1], w[2] };
    ov3 r = scatter_dir(a, mu, u);
    out[0] = r.x; out[1] = r.y; out[2] = r.z;
}

/* Quarter-octave bin of a scatter count: 0 for N=0, else 1 + 4*floor(log2 N) + (two bits below the
 * leading one), capped at 63. */
static int hist_n_bin(uint32_t n)
{
    if (n == 0)
        return 0;
    int e = 31 - __builtin_clz(n);
    int m = (int)((((uint64_t)n << 2) >> e) & 3u);
    int b = 1 + 4 * e + m;
    return b > 63 ? 63 : b;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

typedef struct {
    uint64_t hist_n[64], hist_pos[32 * 64], hist_cos[64], counters[8];
} walk_local;

/* The Eq. 5 term of one event at X (inside the unit sphere) arriving with direction W, toward a point light
 * at xl outside it, per unit light intensity: rho_g(W . w_L) exp(-tau d) / |xl - X|^2 with d the distance
 * from X to the sphere along w_L (the medium fills the sphere of radius 1, optical radius tau). */
static double event_nee(const double* xl, ov3 X, ov3 W, double tau, double g)
{
    ov3 dl = { xl[0] - X.x, xl[1] - X.y, xl[2] - X.z };
    double d2 = dot3(dl, dl);
    double D = sqrt(d2);
    ov3 wl = { dl.x / D, dl.y / D, dl.z / D };
    double b = dot3(X, wl), c = dot3(X, X) - 1.0;
    double disc = b * b - c;
    double d = -b + sqrt(disc > 0.0 ? disc : 0.0);
    double mu = dot3(W, wl);
    double den = 1.0 + g * g - 2.0 * g * mu;
    double rho = (1.0 - g * g) / (4.0 * OM_PI * den * sqrt(den));
    return rho * exp(-tau * d) / d2;
}

static void walk_one(const walk_job* J, uint64_t i, walk_local* L)
{
    const om_medium* m = J->media + (J->per_photon_media ? i : 0);
    uint64_t id = J->photon_offset + i;
    const double sig = m->optical_radius, g = m->g, phi = m->albedo;
    const int paper = m->first_event_at_origin != 0;
    double um[4], ua[4];
    ov3 p = { 0.0, 0.0, 0.0 }, w, x = { 0.0, 0.0, 0.0 };
    ov3 rep_p = { 0.0, 0.0, 0.0 }, rep_w = { 0.0, 0.0, 0.0 };
    int32_t rep_k = 0;
    double pw = 1.0, wsum = 0.0, pe = 1.0, esum = 0.0;
    uint32_t n = 0;
    int status = OM_ESCAPED;

    if (m->isotropic_start) {
        if (paper) {
            draw(J, id, 0u, 1u, ua, NULL);
            w = iso_dir(ua[2], ua[3]);
        } else {
            draw(J, id, 0u, 0u, um, NULL);
            w = iso_dir(um[1], um[2]);
        }
    } else {
        double nn = sqrt(m->dir_in[0] * m->dir_in[0] + m->dir_in[1] * m->dir_in[1] + m->dir_in[2] * m->dir_in[2]);
        w.x = m->dir_in[0] / nn; w.y = m->dir_in[1] / nn; w.z = m->dir_in[2] / nn;
    }

    for (uint32_t s = 0;; ++s) {
        double ures;
        draw(J, id, s, 0u, um, &ures);
        if (s > 0 || paper) {
            /* scattering event at p, arriving with direction w */
            if (n >= J->max_events) {
                status = OM_TRUNCATED;
                break;
            }
            n = n + 1;
            if (J->nee_light) {
                pe = pe * phi;
                esum = esum + pe * event_nee(J->nee_light, p, w, sig, g);
            }
            if (J->reservoir_mode) {
                double wk;
                if (J->reservoir_mode == 1) {
                    wk = 1.0;
                } else {
                    pw = pw * phi;
                    wk = pw;
                }
                wsum = wsum + wk;
                if (ures * wsum < wk) {
                    rep_p = p;
                    rep_w = w;
                    rep_k = (int32_t)n;
                }
            }
            if (J->reservoir_mode != 2 && um[3] >= phi) {
                status = OM_ABSORBED;
                break;
            }
            w = scatter_dir(w, om_hg_cosine(um[1], g), um[2]);
        }
        /* free flight to the next event or to the sphere */
        double l = -om_log(1.0 - um[0]) / sig;
        double b = dot3(p, w);
        double c = dot3(p, p) - 1.0;
        double disc = b * b - c;
        if (disc < 0.0) disc = 0.0;
        double te = -b + sqrt(disc);
        if (l >= te) {
            x.x = p.x + te * w.x; x.y = p.y + te * w.y; x.z = p.z + te * w.z;
            double nx = sqrt(dot3(x, x));
            x.x = x.x / nx; x.y = x.y / nx; x.z = x.z / nx;
            status = OM_ESCAPED;
            break;
        }
        p.x = p.x + l * w.x; p.y = p.y + l * w.y; p.z = p.z + l * w.z;
    }

    L->counters[status] += 1;
    L->counters[3] += n;
    L->hist_n[hist_n_bin(n)] += 1;
    if (status == OM_ESCAPED) {
        int bi = clampi((int)((x.z + 1.0) * 16.0), 0, 31);
        double ph = om_atan2(x.y, x.x);
        int bj = clampi((int)((ph + OM_PI) / OM_2PI * 64.0), 0, 63);
        L->hist_pos[bi * 64 + bj] += 1;
        double mu_out = dot3(w, x);
        L->hist_cos[clampi((int)(mu_out * 64.0), 0, 63)] += 1;
    }
    if (J->n_events) J->n_events[i] = (int32_t)n;
    if (J->status) J->status[i] = (uint8_t)status;
    if (J->exit_pos) {
        J->exit_pos[3 * i] = x.x; J->exit_pos[3 * i + 1] = x.y; J->exit_pos[3 * i + 2] = x.z;
    }
    if (J->exit_dir) {
        ov3 d = status == OM_ESCAPED ? w : (ov3){ 0.0, 0.0, 0.0 };
        J->exit_dir[3 * i] = d.x; J->exit_dir[3 * i + 1] = d.y; J->exit_dir[3 * i + 2] = d.z;
    }
    if (J->rep_pos) {
        J->rep_pos[3 * i] = rep_p.x; J->rep_pos[3 * i + 1] = rep_p.y; J->rep_pos[3 * i + 2] = rep_p.z;
    }
    if (J->rep_dir) {
        J->rep_dir[3 * i] = rep_w.x; J->rep_dir[3 * i + 1] = rep_w.y; J->rep_dir[3 * i + 2] = rep_w.z;
    }
    if (J->rep_index) J->rep_index[i] = rep_k;
    if (J->nee_sum) J->nee_sum[i] = esum;
}

static void* walk_worker(void* arg)
{
    walk_chunk* C = (walk_chunk*)arg;
    walk_local* L = (walk_local*)calloc(1, sizeof(walk_local));
    for (uint64_t i = C->begin; i < C->end; ++i)
        walk_one(C->job, i, L);
    walk_job* J = C->job;
    pthread_mutex_lock(&J->lock);
    for (int k = 0; k < 64; ++k) {
        if (J->hist_n) J->hist_n[k] += L->hist_n[k];
        if (J->hist_cos) J->hist_cos[k] += L->hist_cos[k];
    }
    if (J->hist_pos)
        for (int k = 0; k < 32 * 64; ++k) J->hist_pos[k] += L->hist_pos[k];
    if (J->counters)
        for (int k = 0; k < 8; ++k) J->counters[k] += L->counters[k];
    pthread_mutex_unlock(&J->lock);
    free(L);
    return NULL;
}

/*
 * One walk record: photon `id` of key `seed` in the unit sphere at optical radius tau in the paper's
 * convention (first event at the centre, incoming direction (0,0,1)), following the albedo-1 physics with
 * the representative event chosen with weights phi^k (Sec. 3.2 and Sec. 4.3: the records the three models
 * are trained on).  Outputs N, the exit point x and direction w, the representative event's position X and
 * arriving direction W.  Returns the status (OM_ESCAPED, or OM_TRUNCATED after max_events events).  Used by
 * the renderer's exact-sampler mode, which puts this walk where the three learned samplers would be.
 */
int om_walk_record(uint64_t seed, uint64_t id, double tau, double g, double phi, uint32_t max_events,
                   int32_t* n, double x[3], double w[3], double X[3], double W[3])
{
    om_medium m = { tau, g, phi, { 0.0, 0.0, 1.0 }, 0, 1 };
    uint8_t status = 0;
    int32_t k = 0;
    walk_job J = { seed, id, 1, &m, 0, max_events, 2, 53, n, &status, x, w, X, W, &k,
                   NULL, NULL, NULL, NULL, PTHREAD_MUTEX_INITIALIZER, NULL, NULL };
    walk_local L;
    memset(&L, 0, sizeof(L));
    walk_one(&J, 0, &L);
    return (int)status;
}

/*
 * Run n_photons walks.  Per-photon arrays may be NULL; histograms and counters are accumulated into.
 * counters: [0] escaped, [1] absorbed, [2] truncated, [3] total events, [4..7] zero.
 * Returns the number of threads used.
 */
static int run_walks(walk_job* J, int n_threads)
{
    uint64_t n_photons = J->n_photons;
    int nt = om_num_threads(n_threads);
    if ((uint64_t)nt > n_photons) nt = n_photons > 0 ? (int)n_photons : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    walk_chunk* ch = (walk_chunk*)malloc(sizeof(walk_chunk) * (size_t)nt);
    for (int t = 0; t < nt; ++t) {
        ch[t].job = J;
        ch[t].begin = n_photons * (uint64_t)t / (uint64_t)nt;
        ch[t].end = n_photons * (uint64_t)(t + 1) / (uint64_t)nt;
        pthread_create(&th[t], NULL, walk_worker, &ch[t]);
    }
    for (int t = 0; t < nt; ++t)
        pthread_join(th[t], NULL);
    free(th);
    free(ch);
    return nt;
}

int om_walk(uint64_t seed, uint64_t photon_offset, uint64_t n_photons, const om_medium* media,
            int per_photon_media, uint32_t max_events, int reservoir_mode, int uniform_bits,
            int32_t* n_events, uint8_t* status, double* exit_pos, double* exit_dir, double* rep_pos,
            double* rep_dir, int32_t* rep_index, uint64_t* hist_n, uint64_t* hist_pos, uint64_t* hist_cos,
            uint64_t* counters, int n_threads)
{
    walk_job J = { seed, photon_offset, n_photons, media, per_photon_media, max_events, reservoir_mode,
                   uniform_bits == 24 ? 24 : 53, n_events, status, exit_pos, exit_dir, rep_pos, rep_dir,
                   rep_index, hist_n, hist_pos, hist_cos, counters, PTHREAD_MUTEX_INITIALIZER, NULL, NULL };
    return run_walks(&J, n_threads);
}

/*
 * Walks of the training-record kind (paper convention, incoming direction (0,0,1), albedo-1 physics, the
 * representative event chosen with weights phi^k: reservoir mode 2) that also return, per photon, the
 * brute-force next-event sum over all of its events toward a point light at xl outside the unit sphere,
 * nee_sum[i] = sum_{k=1..N} phi^k rho_g(W_k . w_L) exp(-tau d_k) / |xl - X_k|^2 (Eq. 5: the k-th event's
 * estimate, weighted by the probability phi^(k-1) of reaching it and phi of its own survival term), beside
 * N, the representative event's position, direction and index.  Lets a test compare Lambda^(N) times the
 * representative event's term with the sum on the same walks (Sec. 4.3).  Returns the threads used.
 */
int om_walk_nee(uint64_t seed, uint64_t n_photons, double tau, double g, double phi, const double* xl,
                int32_t* n_events, double* rep_pos, double* rep_dir, int32_t* rep_index, double* nee_sum,
                int n_threads)
{
    om_medium m = { tau, g, phi, { 0.0, 0.0, 1.0 }, 0, 1 };
    walk_job J = { seed, 0, n_photons, &m, 0, 1u << 24, 2, 53, n_events, NULL, NULL, NULL, rep_pos, rep_dir,
                   rep_index, NULL, NULL, NULL, NULL, PTHREAD_MUTEX_INITIALIZER, xl, nee_sum };
    return run_walks(&J, n_threads);
}
