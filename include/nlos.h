/*
 * nlos.h - C ABI of the GB300 (sm_103a) NLOS transient simulator.
 *
 * Implements the forward model of Shi et al., "Fast Non-Line-of-Sight
 * Transient Data Simulation and an Open Benchmark Dataset" (arXiv 2506.03747):
 * the confocal transient integral of the Theory section (Eq. 1; display
 * equations are numbered here in order of appearance), evaluated directly as
 * a sum over (scan point, surface point) pairs and generalised to non-confocal
 * scans, stand-off legs, Lambertian cosines and patch areas; then the
 * detector's Gaussian timing jitter (Eq. 16/17, Algorithm 1 step 2.3) and
 * seeded Poisson photon + dark-count noise (Eq. 18/19, Algorithm 1 step 2.4).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an nlos_status; NLOS_OK is 0. On failure
 *    nlos_last_error() returns a thread-local message (valid until the next
 *    call on that thread). No exception, exit, abort or device trap ever
 *    crosses this boundary.
 *  - "Device pointer" arguments are CUDA global-memory pointers on the current
 *    device; they are caller-owned unless stated otherwise and must be 16-byte
 *    aligned. "cuda_stream" is a cudaStream_t (NULL = legacy default stream).
 *    Work is enqueued asynchronously on that stream unless a call says it
 *    waits.
 *  - Geometry: the relay wall is the plane z = 0 with normal +z, centred at
 *    the origin; hidden surface points have z > 0. The scan grid has
 *    scan_nx x scan_ny cell-centred spots over [-w_x, w_x] x [-w_y, w_y];
 *    scan point s = iy * scan_nx + ix. Transient cubes are float32
 *    [scan_ny][scan_nx][num_bins] (time bin fastest), the paper's
 *    N x N x M layout.
 *  - Point record (float32, 8 per point, "AoS8"): x, y, z, nx, ny, nz,
 *    albedo, area, in metres; (nx, ny, nz) is a unit normal pointing away
 *    from the surface; albedo in [0, 1] (the paper's A/255), area > 0.
 *  - c = 299 792 458 m/s.
 */
#ifndef NLOS_H
#define NLOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NLOS_ABI_VERSION 1

typedef enum {
  NLOS_OK = 0,
  NLOS_EINVAL = 1,      /* bad argument (message says which) */
  NLOS_ENOMEM = 2,      /* device or host allocation failed, or budget refused */
  NLOS_ECUDA = 3,       /* a CUDA runtime call failed */
  NLOS_ETIMEOUT = 4,    /* a bounded device or host wait ran out */
  NLOS_EBUSY = 5,       /* result not ready yet (serving) */
  NLOS_ECANCELLED = 6,  /* request was cancelled (serving) */
  NLOS_ENOTFOUND = 7    /* unknown ticket (serving) */
} nlos_status;

typedef enum { NLOS_CONFOCAL = 0, NLOS_NONCONFOCAL = 1 } nlos_scan_mode;

/* Stand-off (the paper's "stand-off distance", abstract and Introduction):
 * the laser/SPAD optics sit at D = (0, 0, standoff_m) in front of the wall
 * centre. EUCLIDEAN adds the legs |D - l_s| + |d_s - D| to every path;
 * CONSTANT adds 2 * standoff_m (0 gives Eq. 1 exactly, with no device legs). */
typedef enum { NLOS_STANDOFF_EUCLIDEAN = 0, NLOS_STANDOFF_CONSTANT = 1 } nlos_standoff_mode;

/* Cosine terms of the pair weight w = albedo * area * C / (|x-l|^2 |x-d|^2):
 * NONE: C = 1 (Eq. 1 as printed: albedo / r^4 for a confocal scan);
 * OBJECT (default): C = max(0, cos_l) * max(0, cos_d), the Lambertian object
 *   cosines n.(l-x)/|l-x| and n.(d-x)/|d-x| (back-facing patches give no light);
 * OBJECT_WALL: additionally the wall-side cosines (x-l)_z/|x-l| * (x-d)_z/|x-d|. */
typedef enum { NLOS_COS_NONE = 0, NLOS_COS_OBJECT = 1, NLOS_COS_OBJECT_WALL = 2 } nlos_cos_mode;

/* Noise (Eq. 18/19). PEAK: lambda = (peak_photons / max tau_G) * tau_G +
 * dark_per_bin, counts ~ Poisson(lambda). PAPER_NR (Algorithm 1 step 2.4):
 * sigma_n = Var(tau_G) / 10^(nr_db/10) over the whole cube, lambda =
 * sigma_n * tau_G + dark_per_bin; the paper's noisy transient is counts / sigma_n
 * (sigma_n is reported in nlos_stats.noise_scale). */
typedef enum { NLOS_NOISE_NONE = 0, NLOS_NOISE_PEAK = 1, NLOS_NOISE_PAPER_NR = 2 } nlos_noise_mode;

/* NEAREST: bin b = floor(u) of the path-bin coordinate u, then the Gaussian
 * jitter convolution (Algorithm 1: blur, then noise). SPLAT: each pair spreads
 * its weight as w * phi_sigma(b + 1/2 - u) over the bins with
 * |b + 1/2 - u| < 6 sigma (differentiable; no separate blur). */
typedef enum { NLOS_BIN_NEAREST = 0, NLOS_BIN_SPLAT = 1 } nlos_bin_mode;

/* Scene and system parameters (the paper's parameter list: relay surface
 * extent and sampling, stand-off, bin width, acquisition window, jitter FWHM,
 * noise level; abstract, Introduction and Algorithm 1 inputs). */
typedef struct {
  uint32_t struct_size;       /* sizeof(nlos_params), for ABI versioning */
  uint32_t scan_nx, scan_ny;  /* spatial sampling N (>= 1 each) */
  double wall_half_x;         /* w: half side of the scanned area [m] (> 0) */
  double wall_half_y;
  int32_t scan_mode;          /* nlos_scan_mode */
  double laser_x, laser_y;    /* fixed laser spot on the wall (non-confocal) [m] */
  double standoff_m;          /* >= 0 */
  int32_t standoff_mode;      /* nlos_standoff_mode */
  double bin_width_s;         /* Delta t [s] (> 0) */
  uint32_t num_bins;          /* M: bins in the acquisition window (1 .. 65536) */
  double window_start_m;      /* path length at the start of bin 0 [m];
                                 NaN = the device legs of the wall centre
                                 (2 * standoff_m), i.e. t = 0 at the first
                                 bounce on the wall centre, as in Eq. 1 */
  double jitter_fwhm_s;       /* Gaussian jitter FWHM [s]; 0 = none */
  int32_t bin_mode;           /* nlos_bin_mode */
  int32_t cos_mode;           /* nlos_cos_mode */
  int32_t noise_mode;         /* nlos_noise_mode */
  float peak_photons;         /* PEAK mode: expected counts at the cube maximum */
  float dark_per_bin;         /* dark counts added to lambda in every bin */
  float nr_db;                /* PAPER_NR mode: the paper's noise level nr */
  uint64_t seed;              /* Philox key (seed_lo, seed_hi) */
  uint32_t stream_tag;        /* word 3 of every Philox counter */
  float boundary_eps;         /* > 0: count pairs with u within eps of a bin
                                 edge (nlos_stats.boundary_pairs); 0 = off */
  int32_t jitter_padding;     /* boundary rule of the jitter (Eq. 17 gives only
                                 the kernel length): 0 = zero padding (default),
                                 1 = the edge bins continue outside the window
                                 (replicate); NEAREST binning only */
} nlos_params;

/* Fills *p with the defaults: 32x32 confocal scan of a 1 m x 1 m wall, no
 * stand-off, 256 bins of 16 ps, no jitter, COS_OBJECT, no noise. */
void nlos_params_default(nlos_params* p);

typedef struct {
  uint32_t struct_size;       /* set by the caller to sizeof(nlos_stats) */
  uint64_t pairs;             /* scan points x surface points evaluated */
  double peak;                /* max over the cube of tau_G (float32 value) */
  double noise_scale;         /* lambda = noise_scale * tau_G + noise_dark */
  double noise_dark;
  double mean;                /* mean of tau_G over the cube (FP64 sum / n) */
  double variance;            /* population variance of tau_G (FP64) */
  uint64_t boundary_pairs;    /* pairs with u within boundary_eps of a bin edge */
  uint32_t device_error;      /* nonzero: a bounded device wait gave up */
  uint64_t pairs_full;        /* pairs that went through the full per-pair
                                 evaluation, counted per (warp, point pair):
                                 the forward skips, 32 scan points x 2 surface
                                 points at a time, pairs that no lane can bin
                                 (outside the window or facing away), after
                                 computing only r^2 and the cosine numerator */
  uint64_t pairs_tested;      /* pairs of the (scan tile, point block) units
                                 the forward evaluated at all; the others were
                                 ruled out from the bounds of the tile's spots
                                 and of the block's points without touching
                                 the pairs (counted per unit: 32 x 1024) */
} nlos_stats;

typedef struct nlos_scene nlos_scene;

/* Creates a scene: validates the parameters and the points, copies the points
 * to the device and precomputes per-point and per-scan-point terms (FP64 on
 * the device, stored FP32). points_aos8 is host memory when
 * points_on_device == 0, else a device pointer; it is not retained.
 * Points must have finite coordinates, z > 0, area > 0 and albedo >= 0
 * (NLOS_EINVAL otherwise). The call waits for the stream (it checks the
 * points on the device). The library owns the scene's device memory until
 * nlos_scene_destroy. num_points may be 0 (the transient is then zero). */
nlos_status nlos_scene_create(const nlos_params* params, const float* points_aos8,
                              uint64_t num_points, int points_on_device, void* cuda_stream,
                              nlos_scene** out);

/* A scene for the scan rows [row_begin, row_begin + row_count) of the grid
 * that params describes (spots, stand-off legs and window as in the whole
 * grid), for a cube split over devices by scan rows: transients are
 * independent of one another (the jitter section: each scan position is
 * recorded on its own), so each device holds all points and simulates its own
 * rows. Its outputs are [row_count][scan_nx][num_bins]; its Philox streams
 * are those of the global bin indices (row_begin * scan_nx * num_bins + i),
 * so the noise does not depend on the split. nlos_detect on such a scene
 * scales the noise by its own rows; nlos_noise_part scales it by the whole
 * cube. Otherwise as nlos_scene_create (NLOS_EINVAL for an empty or
 * out-of-range row range). */
nlos_status nlos_scene_create_rows(const nlos_params* params, const float* points_aos8,
                                   uint64_t num_points, int points_on_device, uint32_t row_begin,
                                   uint32_t row_count, void* cuda_stream, nlos_scene** out);

/* Replaces the points of a scene by num_points new records (same count as at
 * creation), re-running the ingest/pack step on cuda_stream. Asynchronous:
 * invalid points are reported by the next nlos_simulate with stats
 * (device_error bit 2) or by nlos_scene_check. points_aos8 is host memory
 * (pinned memory keeps the copy asynchronous) when points_on_device == 0. */
nlos_status nlos_scene_set_points(nlos_scene* scene, const float* points_aos8, uint64_t num_points,
                                  int points_on_device, void* cuda_stream);

/* The differentiable parameterisation of the scene (the adjoint's variables,
 * nlos_simulate_backward): point p becomes the record last given to
 * nlos_scene_create / nlos_scene_set_points with its position moved by
 * depth_dev[p] metres along its own unit normal (x + delta n; normal and patch
 * area unchanged) and its albedo replaced by albedo_dev[p]; then the scene is
 * re-ordered and re-packed on the device. albedo_dev, depth_dev: [num_points]
 * float32 device arrays, each nullable (NULL keeps the given albedo / moves
 * nothing). The paper has no such parameterisation (it differentiates
 * nothing); every call starts again from the given records, so calls do not
 * accumulate. Asynchronous; invalid results (albedo < 0, z <= 0) are reported
 * like invalid points (nlos_scene_check, nlos_stats.device_error). The first
 * call allocates a copy of the given records (32 bytes per point). */
nlos_status nlos_scene_set_albedo_depth(nlos_scene* scene, const float* albedo_dev,
                                        const float* depth_dev, void* cuda_stream);

/* Occluders: an extension; the paper's model (Eq. 1) has no visibility term,
 * its depth maps keeping only the first surface seen from the wall. A scene
 * may carry up to NLOS_MAX_OCCLUDERS convex solids, each a record of 8
 * floats {kind, a0, a1, a2, b0, b1, b2, unused}: kind 0 = sphere with centre
 * a and radius b0 > 0, kind 1 = axis-aligned box with corners a < b (per
 * axis). The binned forward then leaves out a pair (s, p) when the segment
 * from its detector spot d_s, or from its laser spot l_s, to the point runs
 * strictly inside some occluder for more than NLOS_OCC_ETA of its length;
 * the tolerance keeps a point on an occluder's own surface visible under
 * FP32 rounding. Non-confocal scans test the laser leg once per point when
 * the points are packed (FP64); the detector leg is tested per pair (FP32).
 * occluders: host memory, copied; count 0 removes them. The points are
 * re-packed on cuda_stream (asynchronous; like every call on a scene, it must
 * not overlap on the device with other work on the same scene), and later
 * forwards use the new set. Serving requests carry no occluders. NLOS_EINVAL: count above
 * NLOS_MAX_OCCLUDERS, an unknown kind, a non-finite value, a radius <= 0 or
 * a box with a >= b on some axis. While a scene has occluders, nlos_forward
 * and nlos_simulate need bin_mode = NLOS_BIN_NEAREST and boundary_eps = 0
 * (NLOS_EINVAL otherwise), and nlos_pair_table ignores them. */
#define NLOS_MAX_OCCLUDERS 16
#define NLOS_OCC_ETA 4e-3f
nlos_status nlos_scene_set_occluders(nlos_scene* scene, const float* occluders, uint32_t count,
                                     void* cuda_stream);

/* Waits for cuda_stream and reports invalid points or a device wait that gave
 * up since the scene was created (NLOS_EINVAL / NLOS_ETIMEOUT). */
nlos_status nlos_scene_check(nlos_scene* scene, void* cuda_stream);

/* Frees the scene (waits for work that uses it on its creation stream). */
nlos_status nlos_scene_destroy(nlos_scene* scene);

/* Number of scan points, bins and points of a scene. */
nlos_status nlos_scene_shape(const nlos_scene* scene, uint64_t* num_scan, uint32_t* num_bins,
                             uint64_t* num_points);

/* The forward pass (the whole hot path) for a scene:
 *   tau_dev    [S][B] float32 device, required: the noise-free transient,
 *              after the jitter convolution (NEAREST) or the splat (SPLAT);
 *   counts_dev [S][B] uint32 device, nullable: Poisson counts (noise_mode !=
 *              NONE; with NONE it must be NULL);
 *   energy_dev [S] double device, nullable: per-transient FP64 sum of tau_dev;
 *   stats      host, nullable: when given, the call waits for the stream and
 *              fills it.
 * Asynchronous on cuda_stream otherwise. Calls on one scene must not overlap
 * on the device (they share its scratch): use one stream per scene.
 * Device memory: the forward's live-unit list (8 bytes a (tile, window, point
 * block) unit) and the noise step's deferred-bin lists (about 3% of the bins)
 * are stream-ordered allocations (cudaMallocAsync) freed on the same stream;
 * the forward returns NLOS_ECUDA when its list cannot be allocated, the noise
 * step falls back to one pass. */
nlos_status nlos_simulate(nlos_scene* scene, float* tau_dev, uint32_t* counts_dev,
                          double* energy_dev, nlos_stats* stats, void* cuda_stream);

/* The two halves of nlos_simulate, for callers that time or overlap them:
 * nlos_forward: the pair histogram with the fused jitter (NEAREST) or the
 *   splat (SPLAT) into tau_dev [S][B] (overwritten);
 * nlos_detect: on a forward result, the per-transient energy (energy_dev,
 *   nullable), the cube maximum / sums and the Poisson counts (counts_dev,
 *   nullable; noise_mode != NONE). Both asynchronous. */
nlos_status nlos_forward(nlos_scene* scene, float* tau_dev, void* cuda_stream);
nlos_status nlos_detect(nlos_scene* scene, const float* tau_dev, uint32_t* counts_dev,
                        double* energy_dev, void* cuda_stream);

/* The noise step (Eq. 18/19, Algorithm 1 step 2.4) of a part of a larger cube
 * (nlos_scene_create_rows): counts_dev [S][B] uint32 ~ Poisson(scale * tau +
 * dark_per_bin) with the scale of the whole cube, computed on the device from
 * cube_stats_dev = {max, sum, sum of squares} of the whole cube's jittered
 * transient (double[3], device: the maximum of the parts' maxima and the sums
 * of their sums, e.g. nlos_reduce's stats combined across devices) and
 * cube_bins, the whole cube's bin count (population variance for PAPER_NR).
 * Asynchronous; NLOS_EINVAL when noise_mode is NONE. */
nlos_status nlos_noise_part(nlos_scene* scene, const float* tau_dev, uint32_t* counts_dev,
                            const double* cube_stats_dev, uint64_t cube_bins, void* cuda_stream);

/* Adjoint of the SPLAT forward (bin_mode must be SPLAT): given grad_tau_dev
 * = dL/dtau ([S][B] float32 device), writes dL/d albedo_p and dL/d delta_p
 * ([P] float32 device each, nullable), where delta_p displaces point p along
 * its normal (normal and area held fixed), evaluated at delta = 0.
 * grad_tau_dev must be 16-byte aligned. Asynchronous on cuda_stream; the
 * outputs are zeroed, then accumulated with global atomics (the order of the
 * FP32 additions, and so the last bits, may differ from call to call).
 * Device memory: for a splat of sigma >= 2.5 bins (the moment form) a
 * stream-ordered table of S x (B + 2J) x 48 bytes, J = ceil(6 sigma) + 1,
 * allocated with cudaMallocAsync and freed on the same stream; NLOS_ECUDA
 * when it cannot be allocated. */
nlos_status nlos_simulate_backward(nlos_scene* scene, const float* grad_tau_dev,
                                   float* grad_albedo_dev, float* grad_depth_dev,
                                   void* cuda_stream);

/* ---- Step-level entry points (each one step of the hot path) ------------ */

/* Gaussian jitter (Eq. 16/17): out[t][b] = sum_j g_j in[t][b - j], j = -R..R,
 * R = ceil(2 sigma), sigma = fwhm_s / (2 sqrt(2 ln 2) bin_width_s), taps
 * exp(-j^2 / (2 sigma^2)) normalised to sum 1, zero padding; fwhm_s = 0 copies.
 * in and out are [num_traces][num_bins] float32 device and must not overlap. */
nlos_status nlos_jitter(const float* in_dev, float* out_dev, uint64_t num_traces,
                        uint32_t num_bins, double fwhm_s, double bin_width_s, void* cuda_stream);

/* nlos_jitter with a boundary rule: padding 0 = zero padding (as nlos_jitter),
 * 1 = replicate (in[b] for b < 0 reads in[0], for b >= num_bins in[num_bins-1]). */
nlos_status nlos_jitter_padded(const float* in_dev, float* out_dev, uint64_t num_traces,
                               uint32_t num_bins, double fwhm_s, double bin_width_s,
                               int32_t padding, void* cuda_stream);

/* Per-trace FP64 energy (energy_dev [num_traces], nullable) and the cube's
 * maximum and FP64 sum / sum of squares (written to stats_dev, nullable:
 * {double max, double sum, double sumsq}). Asynchronous. */
nlos_status nlos_reduce(const float* tau_dev, uint64_t num_traces, uint32_t num_bins,
                        double* energy_dev, double* stats_dev, void* cuda_stream);

/* nlos_reduce without any device allocation. The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory when
 * they call it (their memory is reserved up front by another allocator, such
 * as a framework's caching pool, so a new cudaMalloc may fail; or their loop
 * cannot afford the synchronisation that cudaMalloc/cudaFree may cause).
 * Same arguments and results as nlos_reduce (energy_dev, stats_dev nullable;
 * stats_dev receives {double max, double sum, double sumsq}), computed
 * deterministically (no atomics), asynchronous on cuda_stream.
 * Limit: num_traces <= 65536 (NLOS_EINVAL beyond). The per-transient partial
 * results are kept in a fixed 1.5 MiB array in the library's device image,
 * which every device that loads the library holds until the process exits.
 * The first call on a device looks up that array's device address (once per
 * device, with the device current, and again only if the device's context
 * was destroyed and made anew, e.g. after cudaDeviceReset); make that first
 * call before any stream capture. Every call reuses the array: calls whose work may overlap on the
 * GPU (unordered streams) race on it and must be serialised by the caller. */
nlos_status nlos_reduce_static(const float* tau_dev, uint64_t num_traces, uint32_t num_bins,
                               double* energy_dev, double* stats_dev, void* cuda_stream);

/* Poisson noise (Eq. 18/19): counts[i] ~ Poisson(fmaf(scale, tau[i], dark))
 * for the global bin index j = index_base + i. Draws: key = (seed_lo,
 * seed_hi); bins go in groups of four, and the first uniform of bin j is word
 * (j mod 4) of the Philox4x32-10 block at counter (g_lo, g_hi, 0, stream_tag),
 * g = j / 4; any further uniform comes from the bin's own counters
 * (j_lo, j_hi, 1 + b, stream_tag), b = 0, 1, ..., word after word; a word w
 * gives the uniform ((w >> 9) + 0.5) * 2^-23. Three exact samplers by range:
 * lambda < 30, inversion by sequential search from the first uniform in
 * single precision (p_0 = expf(-lambda), p_k = (p_{k-1} lambda) (1/k),
 * F_k = F_{k-1} + p_k; the first k with u <= F_k, or the first k whose term
 * leaves F unchanged); 30 <= lambda < 150, the sum of ceil(lambda / 30) such
 * draws of mean lambda / ceil(lambda / 30), the first from the first uniform
 * and the others from the own counters (a sum of independent Poisson
 * variables is Poisson); lambda >= 150, Hoermann's PTRS (1993) in double
 * precision on the own counters. lambda <= 0 or NaN gives 0.
 * tau_dev, counts_dev: n floats / uint32 on the device (any alignment; 16-byte
 * alignment with index_base a multiple of 4 takes the vector path).
 * Asynchronous on cuda_stream; NLOS_EINVAL for null pointers with n > 0 and
 * for a scale or dark that is not finite and >= 0. */
nlos_status nlos_noise(const float* tau_dev, uint64_t n, float scale, float dark, uint64_t seed,
                       uint32_t stream_tag, uint64_t index_base, uint32_t* counts_dev,
                       void* cuda_stream);

/* Raw Philox4x32-10 (Salmon et al., SC'11) words: out[i] (4 words) =
 * philox(counter_i, key) for the n counters in ctr_dev ([n][4] uint32
 * device), key = (key0, key1). */
nlos_status nlos_philox(const uint32_t* ctr_dev, uint64_t n, uint32_t key0, uint32_t key1,
                        uint32_t* out_dev, void* cuda_stream);

/* Debug/parity: the forward kernel's own per-pair path-bin coordinate u and
 * weight w (float32, [s_count][P] device each, nullable) for scan points
 * s_begin .. s_begin + s_count - 1, computed by the same device code. */
nlos_status nlos_pair_table(nlos_scene* scene, uint64_t s_begin, uint64_t s_count, float* u_dev,
                            float* w_dev, void* cuda_stream);

/* ---- The paper's FFT forward model (light-cone transform convolution) ---- */

typedef struct nlos_lct nlos_lct;

/* Plan of the paper's FFT forward model (the Theory section's 3-D convolution
 * tau = R_t^{-1} F^{-1}[F(R_z V) . F(PSF)], Algorithm 1 steps 1.1-2.2) for an
 * n x n confocal depth map over a wall of half side wall_half_m, with m time
 * bins of bin_width_s (n, m powers of two; n <= 1024, m <= 4096). Computes the
 * PSF (one node per lateral column, slope = w / (m c dt)) and its 3-D FFT on
 * the zero-padded (2n) x (2n) x (2m) grid; holds two complex FP64 volumes of
 * that size on the device (32 n^2 m bytes each). Synchronous. */
nlos_status nlos_lct_create(uint32_t n, uint32_t m, double wall_half_m, double bin_width_s,
                            void* cuda_stream, nlos_lct** out);

/* One forward pass (asynchronous on cuda_stream, FP64 inside):
 *   depth_dev  [n][n] int32 device: depth bin of each pixel (out of [0, m):
 *              no surface there);
 *   albedo_dev [n][n] float32 device, nullable (NULL: 0.5, as Algorithm 1);
 *   tau_dev    [n][n][m] float32 device, overwritten.
 * Depth bin j (0-based) enters the squared-depth sample ceil((j+1)^2 / m) with
 * weight albedo / ((j+1) m^2); time bin j reads squared-time sample
 * ceil((j+1)^2 / m) times m / (j+1)^4. Calls on one plan must not overlap. */
nlos_status nlos_lct_forward(nlos_lct* plan, const int32_t* depth_dev, const float* albedo_dev,
                             float* tau_dev, void* cuda_stream);

/* Waits for the device and frees the plan. */
nlos_status nlos_lct_destroy(nlos_lct* plan);

/* ---- Serving: continuous batching of simulation requests ---------------- */

typedef struct nlos_server nlos_server;

/* Creates a server that admits requests while the device memory they hold
 * stays within hbm_budget_bytes, and runs their work from one persistent
 * kernel launch per batch. */
nlos_status nlos_server_create(uint64_t hbm_budget_bytes, nlos_server** out);

/* Queues a request (points are host memory, copied); returns its ticket. */
nlos_status nlos_serve_submit(nlos_server* server, const nlos_params* params,
                              const float* points_aos8, uint64_t num_points, uint64_t* ticket_out);

/* Waits up to wait_ms (0 = poll) for a result. NLOS_EBUSY while pending;
 * on NLOS_OK the device pointers (owned by the server, valid until
 * nlos_serve_release) and stats are filled (each output nullable). */
nlos_status nlos_serve_poll(nlos_server* server, uint64_t ticket, int wait_ms,
                            const float** tau_dev_out, const uint32_t** counts_dev_out,
                            nlos_stats* stats);

/* Invalidates the ticket: cancels a pending request, frees a finished one, or
 * (admitted request) frees its memory as soon as its device work completes. */
nlos_status nlos_serve_release(nlos_server* server, uint64_t ticket);

/* Waits (up to 30 s) for admitted requests, cancels pending ones, stops the
 * scheduler and frees everything. */
nlos_status nlos_server_destroy(nlos_server* server);

/* Monitoring: device bytes held by admitted requests, and the numbers of
 * pending and admitted requests (each output nullable). */
nlos_status nlos_server_stats(nlos_server* server, uint64_t* resident_bytes, uint32_t* pending,
                              uint32_t* active);

/* Device time of the serving kernel so far, in SM clock cycles summed over
 * its CTAs (one CTA per SM), updated as its launches end: [0] waiting for or
 * claiming work items, [1] running FORWARD items, [2] running the other
 * items (pack, zero, reduce, noise). For tuning and monitoring; the paper has
 * no counterpart. */
nlos_status nlos_server_device_cycles(nlos_server* server, uint64_t cycles_out[3]);

/* Testing of failure handling, host side only: arms one fault for the next
 * request the scheduler handles. 1 = withhold the publication of its first
 * work item (the device's bounded wait gives up after about a second and the
 * request fails with NLOS_ETIMEOUT, while the server keeps running);
 * 2 = refuse its device allocation (the request fails with NLOS_ENOMEM). */
nlos_status nlos_server_inject(nlos_server* server, int fault);

/* ---- Measurement: throughput of the units the forward is bound by -------- */

/* Element operations per SM clock per SM (clock64 around each timed loop, one
 * 1024-thread CTA per SM), the denominators of the forward's roofline. The
 * paper has no counterpart (it reports no timings); these are the peaks of
 * the GPU the library runs on. Shared reductions use the forward's histogram
 * layout ([row][32] words, lane l on bank l, rows differing per lane). */
typedef struct {
  uint32_t struct_size;       /* set by the caller to sizeof(nlos_peaks) */
  int32_t num_sms;
  double ffma;                /* scalar FP32 fma */
  double ffma2;               /* packed FP32x2 fma (two per lane and instruction) */
  double sqrt_approx;         /* MUFU square root estimate */
  double rcp_approx;          /* MUFU reciprocal estimate */
  double rsqrt_approx;        /* MUFU reciprocal square root estimate */
  double lds128_broadcast;    /* 16-byte shared loads, one address per warp (lanes) */
  double red_f32;             /* red.shared.add.f32, all 32 lanes active */
  double red_u32;             /* red.shared.add.u32, all lanes */
  double red_u64;             /* red.shared.add.u64, all lanes (8-byte words) */
  double rmw_f32;             /* non-atomic shared load + add + store, all lanes */
  double red_f32_quarter;     /* red.shared.add.f32 with one lane in four active */
  double red_u32_quarter;     /* red.shared.add.u32 with one lane in four active */
  double dfma;                /* FP64 fma (the FFT forward model's arithmetic) */
  double atom_f32;            /* atom.shared.add.f32 (old value returned), all lanes */
} nlos_peaks;

/* Runs the microbenchmarks on the current device (about a second; waits for
 * cuda_stream). Allocates a small stream-ordered scratch. */
nlos_status nlos_measure_peaks(nlos_peaks* out, void* cuda_stream);

/* ---- Misc ---------------------------------------------------------------- */

const char* nlos_last_error(void);
int nlos_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NLOS_H */
