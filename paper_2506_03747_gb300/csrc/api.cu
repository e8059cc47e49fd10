// C ABI entry points of the GB300 NLOS simulator (declared in include/nlos.h).
// Argument checking, error reporting and the sequencing of the hot path's
// kernels on the caller's stream; every step of the path runs in this
// library's CUDA kernels.
#include "common.cuh"

#include <cmath>
#include <cstddef>
#include <cstring>
#include <string>

namespace nlos {

nlos_status scene_create(const nlos_params* params, const float* pts, uint64_t P, int on_device,
                         cudaStream_t st, nlos_scene** out);
nlos_status scene_create_rows(const nlos_params* params, const float* pts, uint64_t P,
                              int on_device, uint32_t row_begin, uint32_t row_count,
                              cudaStream_t st, nlos_scene** out);
nlos_status scene_destroy(nlos_scene* sc);
nlos_status scene_set_points(nlos_scene* sc, const float* pts, uint64_t P, int on_device,
                             cudaStream_t st);
nlos_status scene_set_albedo_depth(nlos_scene* sc, const float* albedo, const float* depth,
                                   cudaStream_t st);

namespace {
thread_local std::string g_last_error;
}

nlos_status set_error(nlos_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

nlos_status cuda_error(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return NLOS_ECUDA;
}

void clear_error() { g_last_error.clear(); }

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Global index of the scene's first bin in the whole cube (its Philox streams).
uint64_t first_bin(const Geometry& g) { return (uint64_t)g.row0 * g.nx * g.B; }

}  // namespace

}  // namespace nlos

using namespace nlos;

extern "C" {

void nlos_params_default(nlos_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(nlos_params);
  p->scan_nx = 32;
  p->scan_ny = 32;
  p->wall_half_x = 0.5;
  p->wall_half_y = 0.5;
  p->scan_mode = NLOS_CONFOCAL;
  p->standoff_m = 0.0;
  p->standoff_mode = NLOS_STANDOFF_CONSTANT;
  p->bin_width_s = 16e-12;
  p->num_bins = 256;
  p->window_start_m = NAN;
  p->jitter_fwhm_s = 0.0;
  p->bin_mode = NLOS_BIN_NEAREST;
  p->cos_mode = NLOS_COS_OBJECT;
  p->noise_mode = NLOS_NOISE_NONE;
  p->peak_photons = 100.f;
  p->dark_per_bin = 1e-3f;
  p->nr_db = 2.f;
  p->seed = 0;
  p->stream_tag = 0;
  p->boundary_eps = 0.f;
}

int nlos_abi_version(void) { return NLOS_ABI_VERSION; }

const char* nlos_last_error(void) { return g_last_error.c_str(); }

nlos_status nlos_scene_create(const nlos_params* params, const float* points_aos8,
                              uint64_t num_points, int points_on_device, void* cuda_stream,
                              nlos_scene** out) {
  clear_error();
  try {
    return scene_create(params, points_aos8, num_points, points_on_device, as_stream(cuda_stream),
                        out);
  } catch (...) {
    return set_error(NLOS_ENOMEM, "host exception in nlos_scene_create");
  }
}

nlos_status nlos_scene_destroy(nlos_scene* scene) {
  clear_error();
  return scene_destroy(scene);
}

nlos_status nlos_scene_shape(const nlos_scene* scene, uint64_t* num_scan, uint32_t* num_bins,
                             uint64_t* num_points) {
  clear_error();
  if (!scene) return set_error(NLOS_EINVAL, "scene is NULL");
  if (num_scan) *num_scan = scene->impl.g.S;
  if (num_bins) *num_bins = scene->impl.g.B;
  if (num_points) *num_points = scene->impl.g.P;
  return NLOS_OK;
}

nlos_status nlos_scene_create_rows(const nlos_params* params, const float* points_aos8,
                                   uint64_t num_points, int points_on_device, uint32_t row_begin,
                                   uint32_t row_count, void* cuda_stream, nlos_scene** out) {
  clear_error();
  try {
    return scene_create_rows(params, points_aos8, num_points, points_on_device, row_begin,
                             row_count, as_stream(cuda_stream), out);
  } catch (...) {
    return set_error(NLOS_ENOMEM, "host allocation failed");
  }
}

nlos_status nlos_scene_set_points(nlos_scene* scene, const float* points_aos8, uint64_t num_points,
                                  int points_on_device, void* cuda_stream) {
  clear_error();
  return scene_set_points(scene, points_aos8, num_points, points_on_device, as_stream(cuda_stream));
}

nlos_status nlos_scene_set_albedo_depth(nlos_scene* scene, const float* albedo_dev,
                                       const float* depth_dev, void* cuda_stream) {
  clear_error();
  if ((albedo_dev && !aligned16(albedo_dev)) || (depth_dev && !aligned16(depth_dev)))
    return set_error(NLOS_EINVAL, "albedo_dev and depth_dev must be 16-byte aligned");
  return scene_set_albedo_depth(scene, albedo_dev, depth_dev, as_stream(cuda_stream));
}

nlos_status nlos_scene_set_occluders(nlos_scene* scene, const float* occluders, uint32_t count,
                                     void* cuda_stream) {
  clear_error();
  if (!scene) return set_error(NLOS_EINVAL, "scene is NULL");
  if (count > (uint32_t)kMaxOcc) return set_error(NLOS_EINVAL, "more than NLOS_MAX_OCCLUDERS occluders");
  if (count && !occluders) return set_error(NLOS_EINVAL, "occluders is NULL");
  OccSet o{};
  o.n = (int)count;
  o.eta = NLOS_OCC_ETA;
  for (uint32_t k = 0; k < count; ++k) {
    const float* r = occluders + 8 * k;
    for (int c = 0; c < 7; ++c)
      if (!std::isfinite(r[c])) return set_error(NLOS_EINVAL, "non-finite occluder value");
    if (r[0] == 0.f) {
      if (!(r[4] > 0.f)) return set_error(NLOS_EINVAL, "sphere occluder with radius <= 0");
    } else if (r[0] == 1.f) {
      if (!(r[1] < r[4] && r[2] < r[5] && r[3] < r[6]))
        return set_error(NLOS_EINVAL, "box occluder needs a < b on every axis");
    } else {
      return set_error(NLOS_EINVAL, "unknown occluder kind (0 sphere, 1 box)");
    }
    o.occ[2 * k] = make_float4(r[1], r[2], r[3], r[0]);
    o.occ[2 * k + 1] = make_float4(r[4], r[5], r[6], 0.f);
  }
  SceneImpl& s = scene->impl;
  s.occ = o;
  if (s.g.P == 0) return NLOS_OK;
  NLOS_CUDA_TRY(launch_order_pack(s, as_stream(cuda_stream)));
  return NLOS_OK;
}

nlos_status nlos_scene_check(nlos_scene* scene, void* cuda_stream) {
  clear_error();
  if (!scene) return set_error(NLOS_EINVAL, "scene is NULL");
  cudaStream_t st = as_stream(cuda_stream);
  unsigned int err = 0;
  NLOS_CUDA_TRY(cudaMemcpyAsync(&err, &scene->impl.scratch->err, sizeof(err),
                                cudaMemcpyDeviceToHost, st));
  NLOS_CUDA_TRY(cudaMemsetAsync(&scene->impl.scratch->err, 0, sizeof(err), st));
  NLOS_CUDA_TRY(cudaStreamSynchronize(st));
  if (err & kErrBadPoint)
    return set_error(NLOS_EINVAL, "invalid surface point: need finite values, z > 0, area > 0, "
                                  "albedo >= 0, unit normal");
  if (err & kErrWaitTimeout) return set_error(NLOS_ETIMEOUT, "a bounded device wait gave up");
  return NLOS_OK;
}

nlos_status nlos_forward(nlos_scene* scene, float* tau_dev, void* cuda_stream) {
  clear_error();
  if (!scene) return set_error(NLOS_EINVAL, "scene is NULL");
  SceneImpl& s = scene->impl;
  if (!tau_dev || !aligned16(tau_dev))
    return set_error(NLOS_EINVAL, "tau_dev must be a 16-byte aligned device pointer");
  if (s.occ.n > 0 && (s.g.bin_mode != NLOS_BIN_NEAREST || s.params.boundary_eps > 0.f))
    return set_error(NLOS_EINVAL, "occluders need bin_mode = NLOS_BIN_NEAREST and boundary_eps = 0");
  cudaStream_t st = as_stream(cuda_stream);
  NLOS_CUDA_TRY(cudaMemsetAsync(reinterpret_cast<char*>(s.scratch) + kScratchResetOffset, 0,
                                sizeof(SceneScratch) - kScratchResetOffset, st));
  NLOS_CUDA_TRY(launch_forward(s, tau_dev, st));
  return NLOS_OK;
}

nlos_status nlos_detect(nlos_scene* scene, const float* tau_dev, uint32_t* counts_dev,
                        double* energy_dev, void* cuda_stream) {
  clear_error();
  if (!scene) return set_error(NLOS_EINVAL, "scene is NULL");
  SceneImpl& s = scene->impl;
  const Geometry& g = s.g;
  if (!tau_dev || !aligned16(tau_dev))
    return set_error(NLOS_EINVAL, "tau_dev must be a 16-byte aligned device pointer");
  if (counts_dev && !aligned16(counts_dev))
    return set_error(NLOS_EINVAL, "counts_dev must be 16-byte aligned");
  if (counts_dev && g.noise_mode == NLOS_NOISE_NONE)
    return set_error(NLOS_EINVAL, "counts_dev given but noise_mode is NONE");
  cudaStream_t st = as_stream(cuda_stream);
  // reset the reduction results (not the forward's counters)
  NLOS_CUDA_TRY(cudaMemsetAsync(&s.scratch->peak_bits, 0, sizeof(unsigned int), st));
  NLOS_CUDA_TRY(cudaMemsetAsync(&s.scratch->sum, 0,
                                offsetof(SceneScratch, pairs_full) - offsetof(SceneScratch, sum), st));
  NLOS_CUDA_TRY(launch_reduce(tau_dev, g.S, g.B, energy_dev, s.scratch, st));
  if (counts_dev)
    NLOS_CUDA_TRY(launch_noise_scene(tau_dev, g.S * (uint64_t)g.B, s.scratch, g.noise_mode,
                                     s.params.peak_photons, s.params.dark_per_bin,
                                     s.params.nr_db, s.params.seed, s.params.stream_tag,
                                     counts_dev, st, first_bin(g)));
  return NLOS_OK;
}

nlos_status nlos_noise_part(nlos_scene* scene, const float* tau_dev, uint32_t* counts_dev,
                            const double* cube_stats_dev, uint64_t cube_bins, void* cuda_stream) {
  clear_error();
  if (!scene) return set_error(NLOS_EINVAL, "scene is NULL");
  SceneImpl& s = scene->impl;
  const Geometry& g = s.g;
  if (!tau_dev || !aligned16(tau_dev) || !counts_dev || !aligned16(counts_dev))
    return set_error(NLOS_EINVAL, "tau_dev and counts_dev must be 16-byte aligned device pointers");
  if (!cube_stats_dev) return set_error(NLOS_EINVAL, "cube_stats_dev is NULL");
  if (g.noise_mode == NLOS_NOISE_NONE) return set_error(NLOS_EINVAL, "noise_mode is NONE");
  if (cube_bins < g.S * (uint64_t)g.B)
    return set_error(NLOS_EINVAL, "cube_bins is smaller than the scene's own bins");
  NLOS_CUDA_TRY(launch_noise_scene(tau_dev, g.S * (uint64_t)g.B, s.scratch, g.noise_mode,
                                   s.params.peak_photons, s.params.dark_per_bin, s.params.nr_db,
                                   s.params.seed, s.params.stream_tag, counts_dev,
                                   as_stream(cuda_stream), first_bin(g), cube_stats_dev,
                                   cube_bins));
  return NLOS_OK;
}

nlos_status nlos_simulate(nlos_scene* scene, float* tau_dev, uint32_t* counts_dev,
                          double* energy_dev, nlos_stats* stats, void* cuda_stream) {
  clear_error();
  if (!scene) return set_error(NLOS_EINVAL, "scene is NULL");
  SceneImpl& s = scene->impl;
  const Geometry& g = s.g;
  if (stats && stats->struct_size != sizeof(nlos_stats))
    return set_error(NLOS_EINVAL, "nlos_stats.struct_size does not match this library");
  if (counts_dev && g.noise_mode == NLOS_NOISE_NONE)
    return set_error(NLOS_EINVAL, "counts_dev given but noise_mode is NONE");
  nlos_status r = nlos_forward(scene, tau_dev, cuda_stream);
  if (r != NLOS_OK) return r;
  if (energy_dev || counts_dev || stats) {
    r = nlos_detect(scene, tau_dev, counts_dev, energy_dev, cuda_stream);
    if (r != NLOS_OK) return r;
  }
  if (stats) {
    cudaStream_t st = as_stream(cuda_stream);
    const uint64_t n = g.S * (uint64_t)g.B;
    SceneScratch h{};
    NLOS_CUDA_TRY(cudaMemcpyAsync(&h, s.scratch, sizeof(h), cudaMemcpyDeviceToHost, st));
    NLOS_CUDA_TRY(cudaStreamSynchronize(st));
    stats->pairs = g.S * g.P;
    float peak;
    std::memcpy(&peak, &h.peak_bits, sizeof(peak));
    stats->peak = peak;
    stats->mean = n ? h.sum / (double)n : 0.0;
    stats->variance = n ? h.sumsq / (double)n - stats->mean * stats->mean : 0.0;
    if (stats->variance < 0) stats->variance = 0;
    stats->noise_scale = counts_dev ? h.scale : 0.0;
    stats->noise_dark = counts_dev ? h.dark : 0.0;
    stats->boundary_pairs = h.boundary_pairs;
    stats->device_error = h.err;
    stats->pairs_full = h.pairs_full;
    stats->pairs_tested = h.pairs_tested;
    if (h.err & kErrWaitTimeout) return set_error(NLOS_ETIMEOUT, "a bounded device wait gave up");
    if (h.err & kErrBadPoint) return set_error(NLOS_EINVAL, "invalid surface point (see nlos_scene_check)");
  }
  return NLOS_OK;
}

nlos_status nlos_simulate_backward(nlos_scene* scene, const float* grad_tau_dev,
                                   float* grad_albedo_dev, float* grad_depth_dev,
                                   void* cuda_stream) {
  clear_error();
  if (!scene) return set_error(NLOS_EINVAL, "scene is NULL");
  SceneImpl& s = scene->impl;
  if (s.g.bin_mode != NLOS_BIN_SPLAT)
    return set_error(NLOS_EINVAL, "nlos_simulate_backward needs bin_mode = NLOS_BIN_SPLAT");
  if (!grad_tau_dev || !aligned16(grad_tau_dev))
    return set_error(NLOS_EINVAL, "grad_tau_dev must be a 16-byte aligned device pointer");
  if (!grad_albedo_dev && !grad_depth_dev) return NLOS_OK;
  NLOS_CUDA_TRY(launch_backward(s, grad_tau_dev, grad_albedo_dev, grad_depth_dev,
                                as_stream(cuda_stream)));
  return NLOS_OK;
}

static nlos_status jitter_entry(const float* in_dev, float* out_dev, uint64_t num_traces,
                                uint32_t num_bins, double fwhm_s, double bin_width_s, int padding,
                                void* cuda_stream) {
  clear_error();
  if (!in_dev || !out_dev) return set_error(NLOS_EINVAL, "in_dev and out_dev must not be NULL");
  if (in_dev == out_dev) return set_error(NLOS_EINVAL, "in_dev and out_dev must not overlap");
  if (!(std::isfinite(fwhm_s) && fwhm_s >= 0 && std::isfinite(bin_width_s) && bin_width_s > 0))
    return set_error(NLOS_EINVAL, "fwhm_s must be >= 0 and bin_width_s > 0");
  if (padding != 0 && padding != 1) return set_error(NLOS_EINVAL, "padding must be 0 or 1");
  const double sigma = fwhm_s > 0 ? fwhm_s / (2.0 * std::sqrt(2.0 * std::log(2.0)) * bin_width_s) : 0.0;
  if (jitter_radius(sigma) > 1024) return set_error(NLOS_EINVAL, "jitter kernel radius above 1024 bins");
  NLOS_CUDA_TRY(launch_jitter(in_dev, out_dev, num_traces, num_bins, sigma, padding,
                              as_stream(cuda_stream)));
  return NLOS_OK;
}

nlos_status nlos_jitter(const float* in_dev, float* out_dev, uint64_t num_traces,
                        uint32_t num_bins, double fwhm_s, double bin_width_s, void* cuda_stream) {
  return jitter_entry(in_dev, out_dev, num_traces, num_bins, fwhm_s, bin_width_s, 0, cuda_stream);
}

nlos_status nlos_jitter_padded(const float* in_dev, float* out_dev, uint64_t num_traces,
                               uint32_t num_bins, double fwhm_s, double bin_width_s,
                               int32_t padding, void* cuda_stream) {
  return jitter_entry(in_dev, out_dev, num_traces, num_bins, fwhm_s, bin_width_s, padding,
                      cuda_stream);
}

nlos_status nlos_reduce(const float* tau_dev, uint64_t num_traces, uint32_t num_bins,
                        double* energy_dev, double* stats_dev, void* cuda_stream) {
  clear_error();
  if (!tau_dev) return set_error(NLOS_EINVAL, "tau_dev is NULL");
  if ((num_bins & 3u) == 0u && !aligned16(tau_dev))
    return set_error(NLOS_EINVAL, "tau_dev must be 16-byte aligned");
  cudaStream_t st = as_stream(cuda_stream);
  SceneScratch* scratch = nullptr;
  if (stats_dev) {
    NLOS_CUDA_TRY(cudaMallocAsync(&scratch, sizeof(SceneScratch), st));
    NLOS_CUDA_TRY(cudaMemsetAsync(scratch, 0, sizeof(SceneScratch), st));
  }
  NLOS_CUDA_TRY(launch_reduce(tau_dev, num_traces, num_bins, energy_dev, scratch, st));
  if (stats_dev) {
    // {max, sum, sumsq} as doubles, stream-ordered (no host round trip)
    NLOS_CUDA_TRY(launch_stats_out(scratch, stats_dev, st));
    NLOS_CUDA_TRY(cudaFreeAsync(scratch, st));
  }
  return NLOS_OK;
}

nlos_status nlos_noise(const float* tau_dev, uint64_t n, float scale, float dark, uint64_t seed,
                       uint32_t stream_tag, uint64_t index_base, uint32_t* counts_dev,
                       void* cuda_stream) {
  clear_error();
  if (n && (!tau_dev || !counts_dev)) return set_error(NLOS_EINVAL, "tau_dev and counts_dev must not be NULL");
  if (!(std::isfinite(scale) && scale >= 0 && std::isfinite(dark) && dark >= 0))
    return set_error(NLOS_EINVAL, "scale and dark must be finite and >= 0");
  NLOS_CUDA_TRY(launch_noise(tau_dev, n, scale, dark, seed, stream_tag, index_base, counts_dev,
                             as_stream(cuda_stream)));
  return NLOS_OK;
}

nlos_status nlos_philox(const uint32_t* ctr_dev, uint64_t n, uint32_t key0, uint32_t key1,
                        uint32_t* out_dev, void* cuda_stream) {
  clear_error();
  if (n && (!ctr_dev || !out_dev || !aligned16(ctr_dev) || !aligned16(out_dev)))
    return set_error(NLOS_EINVAL, "ctr_dev and out_dev must be 16-byte aligned device pointers");
  NLOS_CUDA_TRY(launch_philox(ctr_dev, n, key0, key1, out_dev, as_stream(cuda_stream)));
  return NLOS_OK;
}

nlos_status nlos_pair_table(nlos_scene* scene, uint64_t s_begin, uint64_t s_count, float* u_dev,
                            float* w_dev, void* cuda_stream) {
  clear_error();
  if (!scene) return set_error(NLOS_EINVAL, "scene is NULL");
  const Geometry& g = scene->impl.g;
  if (s_begin > g.S || s_count > g.S - s_begin) return set_error(NLOS_EINVAL, "scan range out of bounds");
  NLOS_CUDA_TRY(launch_pair_table(scene->impl, s_begin, s_count, u_dev, w_dev, as_stream(cuda_stream)));
  return NLOS_OK;
}

}  // extern "C"
