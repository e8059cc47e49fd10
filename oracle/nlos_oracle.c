/*
 * FP64 CPU oracle for the NLOS intensity-transport transient simulator
 * (arXiv 2506.03747). TEST INFRASTRUCTURE ONLY: the test suite, the smoke
 * check and the benchmark's CPU-baseline leg use it; the product path never
 * does. It shares no code with the CUDA library.
 *
 * Everything here is the plain definition, evaluated brute force over all
 * (scan point, surface point) pairs, in double precision, with no blocking,
 * fusion or reordering beyond what the definition states. OpenMP only splits
 * independent scan points (or surface points, for the gradient) over threads.
 *
 * Readings of the paper taken here (each restated where it is used):
 *  - c = 299 792 458 m/s (the paper does not state it).
 *  - Scan and surface grids are cell-centred.
 *  - Stand-off: the laser/SPAD optics sit at D = (0, 0, standoff) in front of
 *    the wall centre; the two device legs |D - l_s| + |d_s - D| are part of the
 *    path (or 2*standoff when the constant mode is chosen).
 *  - The acquisition window starts at path length L0 (default: the device legs
 *    of the wall centre, so t = 0 is the first bounce at the wall centre, the
 *    convention of Eq. 1).
 *  - Bin b holds u in [b, b+1); pairs with u < 0 or u >= B are dropped.
 *  - Object-side cosines are clamped at zero (back-facing patches give no
 *    light); no other factor is clamped; no visibility test (Eq. 1 has none)
 *    unless the caller attaches occluders (an extension, see below).
 *  - Jitter taps are normalised to sum 1 and the trace is zero-padded.
 *  - Noise follows Algorithm 1: blur first, then Poisson.
 */
#include "nlos_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------------------
 * Scan geometry.
 * The wall scan is an N_x x N_y grid of spots over [-w_x, w_x] x [-w_y, w_y]
 * (w is the half side of the scanned area, the paper's "w" in Eq. 8). The
 * paper's normalised grid (Eq. 5/6) includes the end points because it serves
 * the padded LCT volume; here each spot sits at the centre of its cell.
 * ------------------------------------------------------------------------- */
void orc_scan_geometry(const orc_geom* g, int64_t s, double l[3], double d[3], double* legs) {
  int64_t ix = s % g->scan_nx;
  int64_t iy = s / g->scan_nx;
  double x = -g->wall_half_x + ((double)ix + 0.5) * (2.0 * g->wall_half_x / (double)g->scan_nx);
  double y = -g->wall_half_y + ((double)iy + 0.5) * (2.0 * g->wall_half_y / (double)g->scan_ny);
  d[0] = x; d[1] = y; d[2] = 0.0;
  if (g->nonconfocal) {
    l[0] = g->laser_x; l[1] = g->laser_y; l[2] = 0.0;
  } else {
    l[0] = x; l[1] = y; l[2] = 0.0;
  }
  if (g->standoff_mode == 1) {
    *legs = 2.0 * g->standoff;
  } else {
    /* device point D = (0, 0, standoff): leg D -> l_s plus leg d_s -> D */
    double a = sqrt(l[0] * l[0] + l[1] * l[1] + g->standoff * g->standoff);
    double b = sqrt(d[0] * d[0] + d[1] * d[1] + g->standoff * g->standoff);
    *legs = a + b;
  }
}

/* Window start L0: explicit, or the device legs of the wall centre (2*standoff). */
double orc_window_start(const orc_geom* g) {
  if (isnan(g->window_start_m)) return 2.0 * g->standoff;
  return g->window_start_m;
}

/* ---------------------------------------------------------------------------
 * One pair (Eq. 1, generalised). The paper's integrand for a confocal scan is
 * rho / r^4 placed at time 2r/c. For a surface sample p with albedo rho_p and
 * patch area a_p, seen from laser spot l and detector spot d:
 *   path   L = legs(s) + |x - l| + |x - d|
 *   bin    u = (L - L0) / (c * dt)
 *   weight w = rho_p * a_p * C / (|x - l|^2 |x - d|^2)
 * with C = 1 (Eq. 1 as printed; gives rho/r^4 when l = d),
 *      C = max(0, cos_l) max(0, cos_d) (Lambertian object, default),
 *      C = the above times the two wall-side cosines (x - l)_z/|x - l| and
 *          (x - d)_z/|x - d|,
 * where cos_l = n . (l - x) / |l - x|, cos_d = n . (d - x) / |d - x|.
 * ------------------------------------------------------------------------- */
static void pair_at(const orc_geom* g, const double l[3], const double d[3], double legs,
                    double L0, const double* pt, double* u, double* w) {
  double vl[3] = {pt[0] - l[0], pt[1] - l[1], pt[2] - l[2]};
  double vd[3] = {pt[0] - d[0], pt[1] - d[1], pt[2] - d[2]};
  double rl = sqrt(vl[0] * vl[0] + vl[1] * vl[1] + vl[2] * vl[2]);
  double rd = sqrt(vd[0] * vd[0] + vd[1] * vd[1] + vd[2] * vd[2]);
  double L = legs + rl + rd;
  *u = (L - L0) / (ORC_LIGHT_SPEED * g->bin_width_s);
  double q = pt[6] * pt[7];
  double C = 1.0;
  if (g->cos_mode >= 1) {
    double cl = -(pt[3] * vl[0] + pt[4] * vl[1] + pt[5] * vl[2]) / rl;
    double cd = -(pt[3] * vd[0] + pt[4] * vd[1] + pt[5] * vd[2]) / rd;
    C = (cl > 0.0 ? cl : 0.0) * (cd > 0.0 ? cd : 0.0);
    if (g->cos_mode == 2) C *= (vl[2] / rl) * (vd[2] / rd);
  }
  *w = q * C / (rl * rl * rd * rd);
}

void orc_pair(const orc_geom* g, int64_t s, const double* pt, double* u, double* w) {
  double l[3], d[3], legs;
  orc_scan_geometry(g, s, l, d, &legs);
  pair_at(g, l, d, legs, orc_window_start(g), pt, u, w);
}

/* ---------------------------------------------------------------------------
 * Binned forward: tau[s][b] = sum of w over pairs with floor(u) = b, 0 <= b < B.
 * Optional outputs for the parity rule of the tests:
 *   flip_mass[s][b]: sum of w over pairs whose u lies within eps of an edge of
 *                    bin b (such a pair may legitimately land on either side in
 *                    a lower-precision evaluation);
 *   edge_mass[s]:    the part of that mass at the window edges u = 0 and u = B;
 *   n_boundary:      the number of pairs within eps of any bin edge 0..B.
 * ------------------------------------------------------------------------- */
int orc_forward_binned(const orc_geom* g, int64_t num_points, const double* pts,
                       int64_t s_begin, int64_t s_count, double* tau,
                       double eps, double* flip_mass, double* edge_mass,
                       int64_t* n_boundary, int num_threads) {
  const int32_t B = g->num_bins;
  const double L0 = orc_window_start(g);
  int64_t nb_total = 0;
  memset(tau, 0, sizeof(double) * (size_t)s_count * (size_t)B);
  if (flip_mass) memset(flip_mass, 0, sizeof(double) * (size_t)s_count * (size_t)B);
  if (edge_mass) memset(edge_mass, 0, sizeof(double) * (size_t)s_count);
#ifdef _OPENMP
  if (num_threads <= 0) num_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(num_threads) reduction(+ : nb_total)
#endif
  for (int64_t i = 0; i < s_count; ++i) {
    double l[3], d[3], legs;
    orc_scan_geometry(g, s_begin + i, l, d, &legs);
    double* row = tau + i * B;
    for (int64_t p = 0; p < num_points; ++p) {
      double u, w;
      pair_at(g, l, d, legs, L0, pts + 8 * p, &u, &w);
      if (u >= 0.0 && u < (double)B) row[(int64_t)floor(u)] += w;
      if (eps > 0.0) {
        double m = floor(u + 0.5);
        if (fabs(u - m) < eps && m >= 0.0 && m <= (double)B) {
          int64_t mi = (int64_t)m;
          nb_total += 1;
          if (flip_mass) {
            if (mi >= 1) flip_mass[i * B + mi - 1] += w;
            if (mi < B) flip_mass[i * B + mi] += w;
          }
          if (edge_mass && (mi == 0 || mi == B)) edge_mass[i] += w;
        }
      }
    }
  }
  if (n_boundary) *n_boundary = nb_total;
  return 0;
}

/* ---------------------------------------------------------------------------
 * Visibility (an extension: the paper's model, Eq. 1, has no visibility term,
 * and its depth maps keep only the first surface seen from the wall).
 * Occluders are convex solids: spheres (centre a, radius b[0]) and
 * axis-aligned boxes (corners a < b). The chord of a segment x -> y through
 * an occluder is the length, in units of the segment, of the set
 *   { t in [0, 1] : x + t (y - x) lies strictly inside the occluder },
 * an interval because the solid is convex. A pair (s, p) is seen when the
 * chord of the segment from each of its spots (laser l_s and detector d_s;
 * one segment when they coincide) to the point is at most eta in every
 * occluder. The tolerance eta (a small fraction of the segment) keeps a
 * point on an occluder's own surface, whose segments leave the solid at
 * once, visible whatever the rounding of its coordinates.
 * ------------------------------------------------------------------------- */
double orc_chord(const orc_occluder* o, const double x[3], const double y[3]) {
  const double d[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
  double t0 = 0.0, t1 = 1.0;
  if (o->kind == 0) {
    /* |x + t d - c|^2 < r^2:  A t^2 + 2 B t + C < 0 */
    const double f[3] = {x[0] - o->a[0], x[1] - o->a[1], x[2] - o->a[2]};
    const double A = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double B = f[0] * d[0] + f[1] * d[1] + f[2] * d[2];
    const double C = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] - o->b[0] * o->b[0];
    if (A == 0.0) return 0.0;
    const double disc = B * B - A * C;
    if (disc <= 0.0) return 0.0;
    const double sq = sqrt(disc);
    const double lo = (-B - sq) / A, hi = (-B + sq) / A;
    if (lo > t0) t0 = lo;
    if (hi < t1) t1 = hi;
  } else {
    /* slabs: a_k < x_k + t d_k < b_k for k = 0, 1, 2 */
    for (int k = 0; k < 3; ++k) {
      if (d[k] == 0.0) {
        if (!(o->a[k] < x[k] && x[k] < o->b[k])) return 0.0;
        continue;
      }
      double ta = (o->a[k] - x[k]) / d[k], tb = (o->b[k] - x[k]) / d[k];
      if (ta > tb) {
        const double tmp = ta;
        ta = tb;
        tb = tmp;
      }
      if (ta > t0) t0 = ta;
      if (tb < t1) t1 = tb;
    }
  }
  return t1 > t0 ? t1 - t0 : 0.0;
}

/* Visibility of point pt from spot z (a point of the wall): 1 if no chord
 * exceeds eta; *border is set when some chord lies within delta of eta. */
static int seen_from(const double z[3], const double* pt, const orc_occluder* occ, int32_t n_occ,
                     double eta, double delta, int* border) {
  int seen = 1;
  for (int32_t k = 0; k < n_occ; ++k) {
    const double c = orc_chord(occ + k, z, pt);
    if (c > eta) seen = 0;
    if (fabs(c - eta) < delta) *border = 1;
  }
  return seen;
}

/* ---------------------------------------------------------------------------
 * Binned forward with occluders: as orc_forward_binned, with each pair's
 * weight kept only when the point is seen from both of its spots. occ_mass
 * (optional) gets, per bin, the weight of in-window pairs whose visibility
 * lies within delta of the threshold (such a pair may legitimately come out
 * either way in a lower-precision evaluation); n_occ_border counts them.
 * ------------------------------------------------------------------------- */
int orc_forward_binned_vis(const orc_geom* g, int64_t num_points, const double* pts,
                           int64_t s_begin, int64_t s_count, const orc_occluder* occ,
                           int32_t n_occ, double eta, double delta, double* tau, double eps,
                           double* flip_mass, double* edge_mass, int64_t* n_boundary,
                           double* occ_mass, int64_t* n_occ_border, int num_threads) {
  const int32_t B = g->num_bins;
  const double L0 = orc_window_start(g);
  int64_t nb_total = 0, no_total = 0;
  memset(tau, 0, sizeof(double) * (size_t)s_count * (size_t)B);
  if (flip_mass) memset(flip_mass, 0, sizeof(double) * (size_t)s_count * (size_t)B);
  if (edge_mass) memset(edge_mass, 0, sizeof(double) * (size_t)s_count);
  if (occ_mass) memset(occ_mass, 0, sizeof(double) * (size_t)s_count * (size_t)B);
#ifdef _OPENMP
  if (num_threads <= 0) num_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(num_threads) reduction(+ : nb_total, no_total)
#endif
  for (int64_t i = 0; i < s_count; ++i) {
    double l[3], d[3], legs;
    orc_scan_geometry(g, s_begin + i, l, d, &legs);
    const int same = l[0] == d[0] && l[1] == d[1] && l[2] == d[2];
    double* row = tau + i * B;
    for (int64_t p = 0; p < num_points; ++p) {
      const double* pt = pts + 8 * p;
      double u, w;
      pair_at(g, l, d, legs, L0, pt, &u, &w);
      int border = 0;
      int seen = 1;
      if (n_occ > 0) {
        seen = seen_from(d, pt, occ, n_occ, eta, delta, &border);
        if (!same) seen = seen_from(l, pt, occ, n_occ, eta, delta, &border) && seen;
      }
      const int in = u >= 0.0 && u < (double)B;
      if (in && seen) row[(int64_t)floor(u)] += w;
      if (border && in && w != 0.0) {
        no_total += 1;
        if (occ_mass) {
          const int64_t b = (int64_t)floor(u);
          occ_mass[i * B + b] += fabs(w);
          /* near a bin edge the pair may also land in the neighbouring bin */
          const double m = floor(u + 0.5);
          if (eps > 0.0 && fabs(u - m) < eps) {
            const int64_t nbr = (int64_t)m == b ? b - 1 : b + 1;
            if (nbr >= 0 && nbr < B) occ_mass[i * B + nbr] += fabs(w);
          }
        }
      }
      if (eps > 0.0 && seen) {
        double m = floor(u + 0.5);
        if (fabs(u - m) < eps && m >= 0.0 && m <= (double)B) {
          int64_t mi = (int64_t)m;
          nb_total += 1;
          if (flip_mass) {
            if (mi >= 1) flip_mass[i * B + mi - 1] += w;
            if (mi < B) flip_mass[i * B + mi] += w;
          }
          if (edge_mass && (mi == 0 || mi == B)) edge_mass[i] += w;
        }
      }
    }
  }
  if (n_boundary) *n_boundary = nb_total;
  if (n_occ_border) *n_occ_border = no_total;
  return 0;
}

/* ---------------------------------------------------------------------------
 * Gaussian timing jitter (Eq. 16/17, Algorithm 1 step 2.3).
 * sigma = FWHM / (2 sqrt(2 ln 2)) expressed in bins, kernel length
 * k = 2 ceil(2 sigma) + 1, taps exp(-j^2 / (2 sigma^2)) normalised to sum 1.
 * FWHM = 0 gives the identity (k = 1). Returns k, or -k if max_taps < k.
 * ------------------------------------------------------------------------- */
int orc_jitter_taps(double fwhm_s, double bin_width_s, double* taps, int max_taps) {
  if (!(fwhm_s > 0.0)) {
    if (max_taps < 1) return -1;
    taps[0] = 1.0;
    return 1;
  }
  double sigma = fwhm_s / (2.0 * sqrt(2.0 * log(2.0)) * bin_width_s);
  int R = (int)ceil(2.0 * sigma);
  int k = 2 * R + 1;
  if (k > max_taps) return -k;
  double sum = 0.0;
  for (int j = -R; j <= R; ++j) {
    taps[j + R] = exp(-(double)j * (double)j / (2.0 * sigma * sigma));
    sum += taps[j + R];
  }
  for (int j = 0; j < k; ++j) taps[j] /= sum;
  return k;
}

/* out[s][b] = sum_j taps[j + R] * tau[s][b - j], j = -R..R, zero outside [0, B). */
void orc_jitter_padded(const double* tau, int64_t num_traces, int32_t num_bins,
                       const double* taps, int32_t k, int32_t padding, double* out) {
  int32_t R = (k - 1) / 2;
  for (int64_t s = 0; s < num_traces; ++s) {
    const double* in = tau + s * num_bins;
    double* o = out + s * num_bins;
    for (int32_t b = 0; b < num_bins; ++b) {
      double acc = 0.0;
      for (int32_t j = -R; j <= R; ++j) {
        int32_t src = b - j;
        if (padding == 1) {  /* replicate: the edge bins continue outside */
          if (src < 0) src = 0;
          if (src > num_bins - 1) src = num_bins - 1;
        }
        if (src >= 0 && src < num_bins) acc += taps[j + R] * in[src];
      }
      o[b] = acc;
    }
  }
}

void orc_jitter(const double* tau, int64_t num_traces, int32_t num_bins,
                const double* taps, int32_t k, double* out) {
  orc_jitter_padded(tau, num_traces, num_bins, taps, k, 0, out);
}

/* ---------------------------------------------------------------------------
 * Philox4x32-10, from Salmon, Moraes, Dror and Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3" (SC'11). Each round multiplies words 0 and 2 of the
 * counter by the two published multipliers, keeps the 64-bit products as
 * (hi, lo) halves, and rebuilds the counter as
 *   (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
 * between rounds the key is bumped by the two published Weyl constants.
 * ------------------------------------------------------------------------- */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += ORC_PHILOX_W0;
      k1 += ORC_PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The same generator over n counters ([n][4] words) under one key (a loop
 * over orc_philox4x32_10, so that tests can compare millions of words). */
void orc_philox_many(const uint32_t* ctr, int64_t n, const uint32_t key[2], uint32_t* out) {
  for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* ---------------------------------------------------------------------------
 * Per-bin random draws, key = (seed_lo, seed_hi). Bins are taken in groups of
 * four, g = floor(index / 4): the first uniform of bin `index` is word
 * (index mod 4) of the block at counter (g_lo, g_hi, 0, stream_tag); any
 * further uniform comes from the bin's own stream, counters
 * (index_lo, index_hi, 1 + j, stream_tag) for j = 0, 1, ..., one word after
 * the other. The group counters have a zero third word and the own-stream
 * counters a nonzero one, so no two draws share a counter. A word w maps to
 * the uniform ((w >> 9) + 0.5) * 2^-23, which lies strictly inside (0, 1) and
 * is exact in single precision.
 * ------------------------------------------------------------------------- */
typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  uint32_t buf[4];
  int pos;
} orc_stream;

static float word_uniform(uint32_t w) { return ((float)(w >> 9) + 0.5f) * 0x1p-23f; }

static float first_uniform(uint64_t index, uint64_t seed, uint32_t stream_tag) {
  const uint64_t g = index >> 2;
  const uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), 0u, stream_tag};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return word_uniform(out[index & 3u]);
}

static void stream_init(orc_stream* st, uint64_t index, uint64_t seed, uint32_t stream_tag) {
  st->key[0] = (uint32_t)seed;
  st->key[1] = (uint32_t)(seed >> 32);
  st->ctr[0] = (uint32_t)index;
  st->ctr[1] = (uint32_t)(index >> 32);
  st->ctr[2] = 1u;
  st->ctr[3] = stream_tag;
  orc_philox4x32_10(st->ctr, st->key, st->buf);
  st->pos = 0;
}

static float stream_uniform(orc_stream* st) {
  if (st->pos == 4) {
    st->ctr[2] += 1u;
    orc_philox4x32_10(st->ctr, st->key, st->buf);
    st->pos = 0;
  }
  return word_uniform(st->buf[st->pos++]);
}

/* ---------------------------------------------------------------------------
 * Poisson sampling (Eq. 18/19). The sampled count decides an integer, so the
 * host and the device take each decision in the same precision: lambda is a
 * single-precision value and the uniforms are exact in single precision;
 *  - lambda < 30: inversion by sequential search in single precision, from
 *    one uniform u: p_0 = expf(-lambda), F_0 = p_0, and for k = 1, 2, ...
 *    p_k = (p_{k-1} lambda) (1/k), F_k = F_{k-1} + p_k, each product, the
 *    reciprocal 1/k and the sum rounded to single precision; the count is
 *    the first k with u <= F_k. The search also stops at the first k whose
 *    term no longer changes F (the single-precision CDF has stopped moving,
 *    a tail of probability ~1e-7), and after 1000 steps;
 *  - 30 <= lambda < 150: the sum of n = ceil(lambda / 30) inversion draws of
 *    mean lambda / n (the first from the bin's first uniform, the others from
 *    its own stream); a sum of independent Poisson variables is Poisson with
 *    the summed mean, so this is exact and keeps every draw in the range
 *    where expf(-mean) is a normal single-precision number;
 *  - lambda >= 150: PTRS, the transformed rejection method with squeeze of
 *    W. Hoermann, "The transformed rejection method for generating Poisson
 *    random variables", Insurance: Mathematics and Economics 12 (1993),
 *    evaluated in double (log and lgamma of double agree to about the last
 *    bit on host and device, where single-precision lgammaf does not), its
 *    uniforms all from the bin's own stream.
 * The PTRS loop is capped at 1000 steps (never reached in practice).
 * lambda <= 0 or NaN gives 0.
 * ------------------------------------------------------------------------- */
static uint32_t poisson_inversion(float lam, float u) {
  float p = expf(-lam);
  float F = p;
  uint32_t k = 0;
  while (u > F && k < 1000u) {
    k += 1u;
    const float rk = 1.0f / (float)k;
    const float q = p * lam;
    p = q * rk;
    const float Fn = F + p;
    if (Fn == F) break;
    F = Fn;
  }
  return k;
}

static uint32_t poisson_ptrs(float lam_f, orc_stream* st) {
  double lam = (double)lam_f;
  double slam = sqrt(lam);
  double loglam = log(lam);
  double b = 0.931 + 2.53 * slam;
  double a = -0.059 + 0.02483 * b;
  double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
  double v_r = 0.9277 - 3.6224 / (b - 2.0);
  for (int it = 0; it < 1000; ++it) {
    double U = (double)stream_uniform(st) - 0.5;
    double V = (double)stream_uniform(st);
    double us = 0.5 - fabs(U);
    double kf = floor((2.0 * a / us + b) * U + lam + 0.43);
    if (us >= 0.07 && V <= v_r) return (uint32_t)kf;
    if (kf < 0.0 || (us < 0.013 && V > us)) continue;
    double lhs = log(V) + log(inv_alpha) - log(a / (us * us) + b);
    double rhs = -lam + kf * loglam - lgamma(kf + 1.0);
    if (lhs <= rhs) return (uint32_t)kf;
  }
  return (uint32_t)floor(lam);
}

uint32_t orc_poisson_one(float lam, uint64_t index, uint64_t seed, uint32_t stream_tag) {
  if (!(lam > 0.0f)) return 0u;
  if (lam < 30.0f) return poisson_inversion(lam, first_uniform(index, seed, stream_tag));
  orc_stream st;
  stream_init(&st, index, seed, stream_tag);
  if (lam < 150.0f) {
    const float parts = ceilf(lam / 30.0f);
    const float sub = lam / parts;
    uint32_t k = poisson_inversion(sub, first_uniform(index, seed, stream_tag));
    for (int i = 1; i < (int)parts; ++i) k += poisson_inversion(sub, stream_uniform(&st));
    return k;
  }
  return poisson_ptrs(lam, &st);
}

void orc_poisson(const float* lam, int64_t n, uint64_t index_base, uint64_t seed,
                 uint32_t stream_tag, uint32_t* counts, int num_threads) {
#ifdef _OPENMP
  if (num_threads <= 0) num_threads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(num_threads)
#endif
  for (int64_t i = 0; i < n; ++i)
    counts[i] = orc_poisson_one(lam[i], index_base + (uint64_t)i, seed, stream_tag);
}

/* ---------------------------------------------------------------------------
 * Differentiable splat (not in the paper, which bins and then blurs): each
 * pair spreads its weight over the bins with a Gaussian of the jitter's sigma,
 *   tau[s][b] = sum_p w_sp * phi(b + 1/2 - u_sp),
 *   phi(x) = exp(-x^2 / (2 sigma^2)) / (sigma sqrt(2 pi)),  |x| < 6 sigma,
 * over bins 0 <= b < B only.
 * ------------------------------------------------------------------------- */
static double splat_kernel(double x, double sigma) {
  return exp(-x * x / (2.0 * sigma * sigma)) / (sigma * sqrt(2.0 * ORC_PI));
}

int orc_forward_splat(const orc_geom* g, double sigma_bins, int64_t num_points,
                      const double* pts, int64_t s_begin, int64_t s_count,
                      double* tau, int num_threads) {
  const int32_t B = g->num_bins;
  const double L0 = orc_window_start(g);
  const double reach = 6.0 * sigma_bins;
  memset(tau, 0, sizeof(double) * (size_t)s_count * (size_t)B);
#ifdef _OPENMP
  if (num_threads <= 0) num_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(num_threads)
#endif
  for (int64_t i = 0; i < s_count; ++i) {
    double l[3], d[3], legs;
    orc_scan_geometry(g, s_begin + i, l, d, &legs);
    double* row = tau + i * B;
    for (int64_t p = 0; p < num_points; ++p) {
      double u, w;
      pair_at(g, l, d, legs, L0, pts + 8 * p, &u, &w);
      /* bins with |b + 1/2 - u| < 6 sigma */
      int64_t b_lo = (int64_t)floor(u - 0.5 - reach);
      int64_t b_hi = (int64_t)ceil(u - 0.5 + reach);
      if (b_lo < 0) b_lo = 0;
      if (b_hi > B - 1) b_hi = B - 1;
      for (int64_t b = b_lo; b <= b_hi; ++b) {
        double x = (double)b + 0.5 - u;
        if (fabs(x) < reach) row[b] += w * splat_kernel(x, sigma_bins);
      }
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Analytic gradient of a loss whose gradient with respect to tau is grad_tau
 * ([S][B], all scan points), through the splat forward above, with respect to
 *   grad_albedo[p] = dL/d rho_p,
 *   grad_depth[p]  = dL/d delta_p at delta = 0, for the displaced point
 *                    x_p + delta * n_p (normal and patch area held fixed).
 * Per pair, with x_b = b + 1/2 - u and phi' = -(x / sigma^2) phi:
 *   G0 = sum_b g[b] phi(x_b),  G1 = sum_b g[b] (x_b / sigma^2) phi(x_b),
 *   dL/d rho   += (dw/d rho) G0,
 *   dL/d delta += (dw/d delta) G0 + w (du/d delta) G1.
 * Leg derivatives (x -> x + delta n):
 *   dr/d delta = -cos,  d cos/d delta = -(1 - cos^2)/r,
 *   d(z/r)/d delta = (n_z + (z/r) cos)/r,  du/d delta = -(cos_l + cos_d)/(c dt).
 * ------------------------------------------------------------------------- */
static void leg_factor(int cos_mode, const double* pt, const double v[3], double r,
                       double* F, double* dF) {
  double ndotv = pt[3] * v[0] + pt[4] * v[1] + pt[5] * v[2];
  double c = -ndotv / r;                 /* cosine at the object */
  double dc = -(1.0 - c * c) / r;        /* its delta-derivative */
  double dr = -c;                        /* d r / d delta */
  double fc = 1.0, dfc = 0.0;            /* cosine factor */
  if (cos_mode >= 1) {
    if (c > 0.0) { fc = c; dfc = dc; } else { fc = 0.0; dfc = 0.0; }
  }
  double fw = 1.0, dfw = 0.0;            /* wall-side cosine factor */
  if (cos_mode == 2) {
    fw = v[2] / r;
    dfw = (pt[5] + fw * c) / r;
  }
  double inv_r2 = 1.0 / (r * r);
  *F = fc * fw * inv_r2;
  *dF = (dfc * fw + fc * dfw) * inv_r2 + fc * fw * (-2.0 * inv_r2 / r) * dr;
}

int orc_backward_splat(const orc_geom* g, double sigma_bins, int64_t num_points,
                       const double* pts, const double* grad_tau,
                       double* grad_albedo, double* grad_depth, int num_threads) {
  const int32_t B = g->num_bins;
  const int64_t S = (int64_t)g->scan_nx * (int64_t)g->scan_ny;
  const double L0 = orc_window_start(g);
  const double cdt = ORC_LIGHT_SPEED * g->bin_width_s;
  const double reach = 6.0 * sigma_bins;
  const double s2 = sigma_bins * sigma_bins;
#ifdef _OPENMP
  if (num_threads <= 0) num_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(num_threads)
#endif
  for (int64_t p = 0; p < num_points; ++p) {
    const double* pt = pts + 8 * p;
    double ga = 0.0, gd = 0.0;
    for (int64_t s = 0; s < S; ++s) {
      double l[3], d[3], legs;
      orc_scan_geometry(g, s, l, d, &legs);
      double vl[3] = {pt[0] - l[0], pt[1] - l[1], pt[2] - l[2]};
      double vd[3] = {pt[0] - d[0], pt[1] - d[1], pt[2] - d[2]};
      double rl = sqrt(vl[0] * vl[0] + vl[1] * vl[1] + vl[2] * vl[2]);
      double rd = sqrt(vd[0] * vd[0] + vd[1] * vd[1] + vd[2] * vd[2]);
      double u = (legs + rl + rd - L0) / cdt;
      double Fl, dFl, Fd, dFd;
      leg_factor(g->cos_mode, pt, vl, rl, &Fl, &dFl);
      leg_factor(g->cos_mode, pt, vd, rd, &Fd, &dFd);
      double q = pt[6] * pt[7];
      double w = q * Fl * Fd;
      double dw_drho = pt[7] * Fl * Fd;
      double dw_ddelta = q * (dFl * Fd + Fl * dFd);
      double cl = -(pt[3] * vl[0] + pt[4] * vl[1] + pt[5] * vl[2]) / rl;
      double cd = -(pt[3] * vd[0] + pt[4] * vd[1] + pt[5] * vd[2]) / rd;
      double du_ddelta = -(cl + cd) / cdt;
      int64_t b_lo = (int64_t)floor(u - 0.5 - reach);
      int64_t b_hi = (int64_t)ceil(u - 0.5 + reach);
      if (b_lo < 0) b_lo = 0;
      if (b_hi > B - 1) b_hi = B - 1;
      double G0 = 0.0, G1 = 0.0;
      const double* grow = grad_tau + s * B;
      for (int64_t b = b_lo; b <= b_hi; ++b) {
        double x = (double)b + 0.5 - u;
        if (fabs(x) < reach) {
          double k = splat_kernel(x, sigma_bins);
          G0 += grow[b] * k;
          G1 += grow[b] * (x / s2) * k;
        }
      }
      ga += dw_drho * G0;
      gd += dw_ddelta * G0 + w * du_ddelta * G1;
    }
    grad_albedo[p] = ga;
    grad_depth[p] = gd;
  }
  return 0;
}

/* Per-pair table for a list of scan points: u[i][p] and w[i][p] as in pair_at. */
void orc_pair_table(const orc_geom* g, int64_t num_points, const double* pts,
                    const int64_t* scan_ids, int64_t n_scan, double* u, double* w,
                    int num_threads) {
  const double L0 = orc_window_start(g);
#ifdef _OPENMP
  if (num_threads <= 0) num_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(num_threads)
#endif
  for (int64_t i = 0; i < n_scan; ++i) {
    double l[3], d[3], legs;
    orc_scan_geometry(g, scan_ids[i], l, d, &legs);
    for (int64_t p = 0; p < num_points; ++p)
      pair_at(g, l, d, legs, L0, pts + 8 * p, u + i * num_points + p, w + i * num_points + p);
  }
}

/* Expected counts per bin in single precision, lambda = fmaf(scale, tau_G, dark)
 * (one rounding), from the double tau_G rounded to float. */
void orc_noise_lambda(const double* tau_g, int64_t n, float scale, float dark, float* lam) {
  for (int64_t i = 0; i < n; ++i) lam[i] = fmaf(scale, (float)tau_g[i], dark);
}
