// Scene creation: parameter and point validation, per-point and per-scan-point
// precomputation (the ingest/pack step of the forward model).
#include "common.cuh"
#include "pack_core.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace nlos {

namespace {

bool finite(double x) { return std::isfinite(x); }

// Validates parameters and resolves the derived geometry.
nlos_status resolve(const nlos_params& p, uint64_t num_points, Geometry& g) {
  if (p.struct_size != sizeof(nlos_params))
    return set_error(NLOS_EINVAL, "nlos_params.struct_size does not match this library");
  if (p.scan_nx < 1 || p.scan_ny < 1 || p.scan_nx > 65536 || p.scan_ny > 65536)
    return set_error(NLOS_EINVAL, "scan_nx and scan_ny must be in 1..65536");
  if (!(finite(p.wall_half_x) && p.wall_half_x > 0 && finite(p.wall_half_y) && p.wall_half_y > 0))
    return set_error(NLOS_EINVAL, "wall_half_x and wall_half_y must be finite and > 0");
  if (p.scan_mode != NLOS_CONFOCAL && p.scan_mode != NLOS_NONCONFOCAL)
    return set_error(NLOS_EINVAL, "scan_mode must be NLOS_CONFOCAL or NLOS_NONCONFOCAL");
  if (!(finite(p.laser_x) && finite(p.laser_y)))
    return set_error(NLOS_EINVAL, "laser_x and laser_y must be finite");
  if (!(finite(p.standoff_m) && p.standoff_m >= 0))
    return set_error(NLOS_EINVAL, "standoff_m must be finite and >= 0");
  if (p.standoff_mode != NLOS_STANDOFF_EUCLIDEAN && p.standoff_mode != NLOS_STANDOFF_CONSTANT)
    return set_error(NLOS_EINVAL, "standoff_mode must be EUCLIDEAN or CONSTANT");
  if (!(finite(p.bin_width_s) && p.bin_width_s > 0))
    return set_error(NLOS_EINVAL, "bin_width_s must be finite and > 0");
  if (p.num_bins < 1 || p.num_bins > 65536)
    return set_error(NLOS_EINVAL, "num_bins must be in 1..65536");
  if (!(std::isnan(p.window_start_m) || finite(p.window_start_m)))
    return set_error(NLOS_EINVAL, "window_start_m must be finite or NaN");
  if (!(finite(p.jitter_fwhm_s) && p.jitter_fwhm_s >= 0))
    return set_error(NLOS_EINVAL, "jitter_fwhm_s must be finite and >= 0");
  if (p.bin_mode != NLOS_BIN_NEAREST && p.bin_mode != NLOS_BIN_SPLAT)
    return set_error(NLOS_EINVAL, "bin_mode must be NEAREST or SPLAT");
  if (p.cos_mode < NLOS_COS_NONE || p.cos_mode > NLOS_COS_OBJECT_WALL)
    return set_error(NLOS_EINVAL, "cos_mode must be NONE, OBJECT or OBJECT_WALL");
  if (p.noise_mode < NLOS_NOISE_NONE || p.noise_mode > NLOS_NOISE_PAPER_NR)
    return set_error(NLOS_EINVAL, "noise_mode must be NONE, PEAK or PAPER_NR");
  if (!(std::isfinite(p.peak_photons) && p.peak_photons >= 0 && std::isfinite(p.dark_per_bin) &&
        p.dark_per_bin >= 0 && std::isfinite(p.nr_db)))
    return set_error(NLOS_EINVAL, "peak_photons, dark_per_bin must be finite and >= 0; nr_db finite");
  if (!(std::isfinite(p.boundary_eps) && p.boundary_eps >= 0 && p.boundary_eps < 0.5f))
    return set_error(NLOS_EINVAL, "boundary_eps must be in [0, 0.5)");
  if (p.jitter_padding != 0 && p.jitter_padding != 1)
    return set_error(NLOS_EINVAL, "jitter_padding must be 0 (zero) or 1 (replicate)");
  if (num_points > (uint64_t)1 << 31)
    return set_error(NLOS_EINVAL, "num_points must be <= 2^31");

  g.nx = p.scan_nx;
  g.ny = p.scan_ny;
  g.row0 = 0;
  g.ny_full = p.scan_ny;
  g.B = p.num_bins;
  g.S = (uint64_t)p.scan_nx * p.scan_ny;
  g.P = num_points;
  g.scan_mode = p.scan_mode;
  g.cos_mode = p.cos_mode;
  g.bin_mode = p.bin_mode;
  g.noise_mode = p.noise_mode;
  g.cdt = kLightSpeed * p.bin_width_s;
  g.L0 = std::isnan(p.window_start_m) ? 2.0 * p.standoff_m : p.window_start_m;
  // sigma in bins: FWHM / (2 sqrt(2 ln 2)) / dt (Algorithm 1 inputs)
  g.sigma = p.jitter_fwhm_s > 0 ? p.jitter_fwhm_s / (2.0 * std::sqrt(2.0 * std::log(2.0)) *
                                                      p.bin_width_s)
                                : 0.0;
  if (p.bin_mode == NLOS_BIN_SPLAT && !(g.sigma >= 0.25))
    return set_error(NLOS_EINVAL, "SPLAT needs a jitter FWHM of at least 0.59 bins (sigma >= 0.25 bins)");
  if (p.bin_mode == NLOS_BIN_NEAREST && jitter_radius(g.sigma) > 64)
    return set_error(NLOS_EINVAL, "jitter sigma above 32 bins is not supported (kernel radius > 64)");
  if (p.bin_mode == NLOS_BIN_SPLAT && 6.0 * g.sigma > 4096)
    return set_error(NLOS_EINVAL, "jitter sigma too wide for SPLAT");
  if (g.S * (uint64_t)g.B > ((uint64_t)1 << 40))
    return set_error(NLOS_EINVAL, "scan_nx * scan_ny * num_bins too large");
  return NLOS_OK;
}


// Per-scan-point spot and bin offset off_s = (legs(s) - L0) / (c dt), FP64.
void scan_points(const nlos_params& p, const Geometry& g, std::vector<ScanPoint>& out) {
  out.resize(g.S);
  const double h = p.standoff_m;
  for (uint64_t s = 0; s < g.S; ++s) {
    const uint64_t ix = s % g.nx, iy = g.row0 + s / g.nx;  // row of the full grid
    const double dx = -p.wall_half_x + ((double)ix + 0.5) * (2.0 * p.wall_half_x / g.nx);
    const double dy = -p.wall_half_y + ((double)iy + 0.5) * (2.0 * p.wall_half_y / g.ny_full);
    const double lx = p.scan_mode == NLOS_NONCONFOCAL ? p.laser_x : dx;
    const double ly = p.scan_mode == NLOS_NONCONFOCAL ? p.laser_y : dy;
    double legs;
    if (p.standoff_mode == NLOS_STANDOFF_CONSTANT) {
      legs = 2.0 * h;
    } else {
      legs = std::sqrt(lx * lx + ly * ly + h * h) + std::sqrt(dx * dx + dy * dy + h * h);
    }
    ScanPoint sp;
    sp.sx = (float)dx;
    sp.sy = (float)dy;
    sp.off = (float)((legs - g.L0) / g.cdt);
    sp.row = (uint32_t)s;
    out[s] = sp;
  }
}

}  // namespace

void compact_tile_order(const std::vector<ScanPoint>& plain, uint32_t nx, uint32_t ny,
                        std::vector<ScanPoint>& out) {
  constexpr uint32_t kPx = 8, kPy = 4;  // kPx * kPy == kTile
  static_assert(kPx * kPy == (uint32_t)kTile, "tile patch");
  out.clear();
  out.reserve(plain.size());
  for (uint32_t py = 0; py < ny; py += kPy)
    for (uint32_t px = 0; px < nx; px += kPx)
      for (uint32_t y = py; y < std::min(ny, py + kPy); ++y)
        for (uint32_t x = px; x < std::min(nx, px + kPx); ++x)
          out.push_back(plain[(uint64_t)y * nx + x]);
}

nlos_status resolve_params(const nlos_params& p, uint64_t num_points, Geometry& g) {
  return resolve(p, num_points, g);
}

// The forward's scan table (tile order).
void scan_points_host(const nlos_params& p, const Geometry& g, std::vector<ScanPoint>& out) {
  std::vector<ScanPoint> plain;
  scan_points(p, g, plain);
  compact_tile_order(plain, g.nx, g.ny, out);
}

nlos_status scene_create_rows(const nlos_params* params, const float* pts, uint64_t P,
                              int on_device, uint32_t row_begin, uint32_t row_count,
                              cudaStream_t st, nlos_scene** out) {
  if (!params || !out) return set_error(NLOS_EINVAL, "params and out must not be NULL");
  *out = nullptr;
  if (P > 0 && !pts) return set_error(NLOS_EINVAL, "points_aos8 is NULL");
  Geometry g{};
  nlos_status rs = resolve(*params, P, g);
  if (rs != NLOS_OK) return rs;
  if (row_count == 0 || (uint64_t)row_begin + row_count > params->scan_ny)
    return set_error(NLOS_EINVAL, "rows [row_begin, row_begin + row_count) must be a non-empty "
                                  "range of the scan_ny rows");
  g.row0 = row_begin;
  g.ny = row_count;
  g.S = (uint64_t)g.nx * row_count;

  nlos_scene* sc = new (std::nothrow) nlos_scene();
  if (!sc) return set_error(NLOS_ENOMEM, "host allocation failed");
  SceneImpl& s = sc->impl;
  s.params = *params;
  s.g = g;
  s.stream = st;
  auto fail = [&](nlos_status code, const std::string& msg) {
    for (void* q : {(void*)s.pairs, (void*)s.scan, (void*)s.scan_fwd, (void*)s.scratch,
                    (void*)s.raw_points,
                    (void*)s.perm, (void*)s.cell, (void*)s.cells, (void*)s.bounds, (void*)s.tiles})
      if (q) cudaFree(q);
    delete sc;
    return set_error(code, msg);
  };
  cudaError_t e = cudaGetDevice(&s.device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, s.device);
  if (e != cudaSuccess) return fail(NLOS_ECUDA, cudaGetErrorString(e));

  const uint64_t n_pairs = (P + 1) / 2;
  const uint64_t n_sub = (n_pairs + kSubPairs - 1) / kSubPairs;
  std::vector<ScanPoint> hs, hf;
  scan_points(*params, g, hs);
  compact_tile_order(hs, g.nx, g.ny, hf);
  std::vector<TileBound> ht;
  tile_bounds_host(hf.data(), g.S, ht);
  if ((e = cudaMalloc(&s.scratch, sizeof(SceneScratch))) != cudaSuccess ||
      (e = cudaMalloc(&s.scan, sizeof(ScanPoint) * (g.S ? g.S : 1))) != cudaSuccess ||
      (e = cudaMalloc(&s.scan_fwd, sizeof(ScanPoint) * (g.S ? g.S : 1))) != cudaSuccess ||
      (e = cudaMalloc(&s.tiles, sizeof(TileBound) * (ht.empty() ? 1 : ht.size()))) != cudaSuccess ||
      (P > 0 && (e = cudaMalloc(&s.pairs, sizeof(PointPair) * n_pairs)) != cudaSuccess) ||
      (P > 0 && (e = cudaMalloc(&s.raw_points, sizeof(float) * 8 * P)) != cudaSuccess) ||
      (P > 0 && (e = cudaMalloc(&s.perm, sizeof(uint32_t) * P)) != cudaSuccess) ||
      (P > 0 && (e = cudaMalloc(&s.cell, sizeof(uint16_t) * P)) != cudaSuccess) ||
      (P > 0 && (e = cudaMalloc(&s.cells, sizeof(uint32_t) * (kOrderCells + 8))) != cudaSuccess) ||
      (P > 0 && (e = cudaMalloc(&s.bounds, sizeof(BlockBound) * n_sub)) != cudaSuccess))
    return fail(NLOS_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));

  e = cudaMemsetAsync(s.scratch, 0, sizeof(SceneScratch), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s.scan, hs.data(), sizeof(ScanPoint) * g.S, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s.scan_fwd, hf.data(), sizeof(ScanPoint) * g.S, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !ht.empty())
    e = cudaMemcpyAsync(s.tiles, ht.data(), sizeof(TileBound) * ht.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && P > 0)
    e = cudaMemcpyAsync(s.raw_points, pts, sizeof(float) * 8 * P,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && P > 0) e = launch_order_pack(s, st);
  unsigned int err = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&err, &s.scratch->err, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(NLOS_ECUDA, cudaGetErrorString(e));
  if (err & kErrBadPoint)
    return fail(NLOS_EINVAL,
                "invalid surface point: need finite values, z > 0, area > 0, albedo >= 0, unit normal");
  *out = sc;
  return NLOS_OK;
}

nlos_status scene_create(const nlos_params* params, const float* pts, uint64_t P, int on_device,
                         cudaStream_t st, nlos_scene** out) {
  return scene_create_rows(params, pts, P, on_device, 0, params ? params->scan_ny : 0, st, out);
}

nlos_status scene_set_points(nlos_scene* sc, const float* pts, uint64_t P, int on_device,
                             cudaStream_t st) {
  if (!sc) return set_error(NLOS_EINVAL, "scene is NULL");
  SceneImpl& s = sc->impl;
  if (P != s.g.P) return set_error(NLOS_EINVAL, "num_points differs from the scene's point count");
  if (P == 0) return NLOS_OK;
  if (!pts) return set_error(NLOS_EINVAL, "points_aos8 is NULL");
  cudaError_t e = cudaMemcpyAsync(s.raw_points, pts, sizeof(float) * 8 * P,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  // the records as given are also the base of later albedo/depth updates
  if (e == cudaSuccess && s.base_points)
    e = cudaMemcpyAsync(s.base_points, s.raw_points, sizeof(float) * 8 * P,
                        cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(points)");
  e = launch_order_pack(s, st);
  if (e != cudaSuccess) return cuda_error(e, "order/pack kernels");
  return NLOS_OK;
}

namespace {

// The differentiable parameterisation of a scene (albedo and normal-offset
// depth): record p = base record p with its position moved by depth[p] along
// its (fixed, unit) normal, x + delta n, and its albedo replaced by albedo[p];
// normal and patch area unchanged. Either array may be null (kept / no move).
__global__ void displace_kernel(const float* __restrict__ base, uint64_t P,
                                const float* __restrict__ albedo, const float* __restrict__ depth,
                                float* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    const float4* b = reinterpret_cast<const float4*>(base + 8 * p);
    float4 r0 = b[0], r1 = b[1];  // (x, y, z, nx), (ny, nz, albedo, area)
    if (depth) {
      const float d = depth[p];
      r0.x = fmaf(d, r0.w, r0.x);
      r0.y = fmaf(d, r1.x, r0.y);
      r0.z = fmaf(d, r1.y, r0.z);
    }
    if (albedo) r1.z = albedo[p];
    float4* o = reinterpret_cast<float4*>(out + 8 * p);
    o[0] = r0;
    o[1] = r1;
  }
}

}  // namespace

nlos_status scene_set_albedo_depth(nlos_scene* sc, const float* albedo, const float* depth,
                                   cudaStream_t st) {
  if (!sc) return set_error(NLOS_EINVAL, "scene is NULL");
  SceneImpl& s = sc->impl;
  const uint64_t P = s.g.P;
  if (P == 0) return NLOS_OK;
  cudaError_t e = cudaSuccess;
  if (!s.base_points) {
    // first use: keep the records as given (raw_points holds them until now)
    if ((e = cudaMalloc(&s.base_points, sizeof(float) * 8 * P)) != cudaSuccess) {
      s.base_points = nullptr;
      return set_error(NLOS_ENOMEM, std::string("device allocation failed: ") +
                                        cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(s.base_points, s.raw_points, sizeof(float) * 8 * P,
                        cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(base points)");
  }
  const uint64_t want = (P + 255) / 256;
  const unsigned grid = (unsigned)std::min<uint64_t>(want, (uint64_t)s.num_sms * 8);
  displace_kernel<<<grid, 256, 0, st>>>(s.base_points, P, albedo, depth, s.raw_points);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_order_pack(s, st);
  if (e != cudaSuccess) return cuda_error(e, "displace/order/pack kernels");
  return NLOS_OK;
}

nlos_status scene_destroy(nlos_scene* sc) {
  if (!sc) return set_error(NLOS_EINVAL, "scene is NULL");
  SceneImpl& s = sc->impl;
  cudaStreamSynchronize(s.stream);
  cudaError_t e = cudaSuccess, e2;
  if (s.pairs && (e2 = cudaFree(s.pairs)) != cudaSuccess) e = e2;
  if (s.scan && (e2 = cudaFree(s.scan)) != cudaSuccess) e = e2;
  if (s.scan_fwd && (e2 = cudaFree(s.scan_fwd)) != cudaSuccess) e = e2;
  if (s.scratch && (e2 = cudaFree(s.scratch)) != cudaSuccess) e = e2;
  if (s.raw_points && (e2 = cudaFree(s.raw_points)) != cudaSuccess) e = e2;
  if (s.base_points && (e2 = cudaFree(s.base_points)) != cudaSuccess) e = e2;
  for (void* q : {(void*)s.perm, (void*)s.cell, (void*)s.cells, (void*)s.bounds, (void*)s.tiles})
    if (q && (e2 = cudaFree(q)) != cudaSuccess) e = e2;
  delete sc;
  if (e != cudaSuccess) return cuda_error(e, "cudaFree");
  return NLOS_OK;
}

}  // namespace nlos
