/*
 * FP64 CPU oracle for the NLOS intensity-transport transient simulator
 * (Shi et al., "Fast Non-Line-of-Sight Transient Data Simulation and an Open
 * Benchmark Dataset", arXiv 2506.03747).
 *
 * TEST INFRASTRUCTURE ONLY. This code is used by the test suite, by the smoke
 * check and by the benchmark's CPU-baseline leg. The product path never links,
 * loads or calls it, and it shares no code, header, table or helper with the
 * CUDA library.
 *
 * Display equations of the paper are unnumbered; they are cited here as
 * Eq. 1 .. Eq. 19 in their order of appearance (Eq. 1 = the confocal transient
 * integral of the Theory section, Eq. 16/17 = the jitter model, Eq. 18/19 =
 * the Poisson noise model), and Algorithm 1 is the "Non-line-of-sight
 * Simulation Pipeline".
 *
 * Point record (double, 8 per point): x, y, z, nx, ny, nz, albedo, area.
 * The relay wall is the plane z = 0 with normal +z; hidden points have z > 0.
 * Scan point index s = iy * scan_nx + ix (row-major), transient layout
 * [s][bin] with the bin index fastest.
 */
#ifndef NLOS_ORACLE_H
#define NLOS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_LIGHT_SPEED 299792458.0 /* m/s; the paper does not state c */

typedef struct {
  int32_t scan_nx, scan_ny;      /* spatial sampling of the relay wall */
  double wall_half_x, wall_half_y; /* w: half side of the scanned area [m] */
  int32_t nonconfocal;           /* 0: laser spot == detector spot */
  double laser_x, laser_y;       /* fixed laser spot on the wall (non-confocal) */
  double standoff;               /* device distance from the wall centre [m] */
  int32_t standoff_mode;         /* 0: Euclidean legs, 1: constant 2*standoff */
  double bin_width_s;            /* Delta t [s] */
  int32_t num_bins;              /* number of time bins B */
  double window_start_m;         /* path length at the start of bin 0; NaN -> default */
  int32_t cos_mode;              /* 0: none (Eq. 1 as printed), 1: object, 2: object + wall */
} orc_geom;

/* Scan geometry: laser spot l_s, detector spot d_s and stand-off legs of scan point s. */
void orc_scan_geometry(const orc_geom* g, int64_t s, double l[3], double d[3], double* legs);
double orc_window_start(const orc_geom* g);

/* Path-bin coordinate u and weight w of one (scan point, surface point) pair. */
void orc_pair(const orc_geom* g, int64_t s, const double* pt, double* u, double* w);

/* Per-pair table u[i][p], w[i][p] for the scan points scan_ids[0..n_scan). */
void orc_pair_table(const orc_geom* g, int64_t num_points, const double* pts,
                    const int64_t* scan_ids, int64_t n_scan, double* u, double* w,
                    int num_threads);

/* Binned forward transient (Eq. 1 discretised on surface samples). */
int orc_forward_binned(const orc_geom* g, int64_t num_points, const double* pts,
                       int64_t s_begin, int64_t s_count, double* tau,
                       double eps, double* flip_mass, double* edge_mass,
                       int64_t* n_boundary, int num_threads);

/* Occluders (an extension; the paper's model has no visibility term):
 * kind 0 = sphere (a = centre, b[0] = radius), kind 1 = axis-aligned box
 * (corners a < b). */
typedef struct {
  int32_t kind;
  double a[3], b[3];
} orc_occluder;

/* Length, in units of the segment, of the part of segment x -> y strictly
 * inside the occluder. */
double orc_chord(const orc_occluder* o, const double x[3], const double y[3]);

/* Binned forward with the pairs whose point is hidden from one of its spots
 * (a chord above eta) left out; occ_mass / n_occ_border: pairs whose chord
 * lies within delta of eta. */
int orc_forward_binned_vis(const orc_geom* g, int64_t num_points, const double* pts,
                           int64_t s_begin, int64_t s_count, const orc_occluder* occ,
                           int32_t n_occ, double eta, double delta, double* tau, double eps,
                           double* flip_mass, double* edge_mass, int64_t* n_boundary,
                           double* occ_mass, int64_t* n_occ_border, int num_threads);

/* Gaussian jitter (Eq. 16/17). */
int orc_jitter_taps(double fwhm_s, double bin_width_s, double* taps, int max_taps);
void orc_jitter(const double* tau, int64_t num_traces, int32_t num_bins,
                const double* taps, int32_t k, double* out);
/* The same with a boundary rule: padding 0 = zero padding (Eq. 17 fixes only
 * k; zero padding is the default reading), 1 = replicate the edge bins. */
void orc_jitter_padded(const double* tau, int64_t num_traces, int32_t num_bins,
                       const double* taps, int32_t k, int32_t padding, double* out);

/* Philox4x32-10 (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox_many(const uint32_t* ctr, int64_t n, const uint32_t key[2], uint32_t* out);

/* Poisson noise (Eq. 18/19, Algorithm 1 step 2.4). */
void orc_noise_lambda(const double* tau_g, int64_t n, float scale, float dark, float* lam);
uint32_t orc_poisson_one(float lam, uint64_t index, uint64_t seed, uint32_t stream_tag);
void orc_poisson(const float* lam, int64_t n, uint64_t index_base, uint64_t seed,
                 uint32_t stream_tag, uint32_t* counts, int num_threads);

/* Differentiable Gaussian-splat forward and its analytic gradient. */
int orc_forward_splat(const orc_geom* g, double sigma_bins, int64_t num_points,
                      const double* pts, int64_t s_begin, int64_t s_count,
                      double* tau, int num_threads);
int orc_backward_splat(const orc_geom* g, double sigma_bins, int64_t num_points,
                       const double* pts, const double* grad_tau,
                       double* grad_albedo, double* grad_depth, int num_threads);

#ifdef __cplusplus
}
#endif
#endif
