/*
 * Oracle internal header — TEST INFRASTRUCTURE ONLY.
 *
 * This is the plain, slow, FP64 CPU restatement of the method that the CUDA path is checked against.
 * Only tests, the smoke check and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, constant table or helper with the CUDA library: the two are written separately from the paper
 * and from the published definitions they cite.
 */
#ifndef MS_ORACLE_H
#define MS_ORACLE_H
#include <stdint.h>

typedef struct { double x, y, z; } ov3;

/* Counter-based generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void om_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void om_philox_words(uint64_t seed, uint64_t id0, uint64_t n_ids, uint32_t step, uint32_t tag, uint32_t* out);

/* Deterministic FP64 functions built from IEEE basic operations only (see detmath.c). */
double om_log(double x);
void om_sincos_turns(double u, double* s, double* c);
double om_atan2(double y, double x);

/* Medium of one walk: Sec. 3.1 (optical radius sigma_t*R, albedo phi, HG g, incoming direction). */
typedef struct {
    double optical_radius, g, albedo;
    double dir_in[3];
    int32_t isotropic_start;        /* 1: initial direction uniform on the sphere                    */
    int32_t first_event_at_origin;  /* 1: first scattering event at the centre (Sec. 3.1 convention) */
} om_medium;

int om_num_threads(int requested);
double om_hg_cosine(double u, double g);
void om_scatter_dir(const double* w, double mu, double u, double* out);

#endif
