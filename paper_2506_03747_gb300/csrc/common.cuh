// Internal declarations of the GB300 NLOS simulator library (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nlos.h"

namespace nlos {

constexpr double kLightSpeed = 299792458.0;
constexpr int kTile = 32;  // scan points per forward tile (one per lane)

// ---------------------------------------------------------------------------
// Error reporting (thread-local message behind nlos_last_error()).
// ---------------------------------------------------------------------------
nlos_status set_error(nlos_status st, const std::string& msg);
nlos_status cuda_error(cudaError_t e, const char* what);
void clear_error();

#define NLOS_CUDA_TRY(expr)                                     \
  do {                                                          \
    cudaError_t _e = (expr);                                    \
    if (_e != cudaSuccess) return ::nlos::cuda_error(_e, #expr); \
  } while (0)

// Device-side status word bits (scene scratch).
constexpr uint32_t kErrWaitTimeout = 1u;   // a bounded mbarrier wait gave up
constexpr uint32_t kErrBadPoint = 2u;      // point validation failed

// ---------------------------------------------------------------------------
// Packed surface points, two per record, interleaved component-wise
// (.x = point 2k, .y = point 2k + 1), 64 bytes:
//   px, py      position x, y
//   pz2         z^2
//   kq          weight factor (cosine-free modes)
//   na, nb, nc  cosine numerator na*(px - sx) + nb*(py - sy) + nc at scan spot
//               (sx, sy, 0), i.e. n.(spot - x) = -(nx dx + ny dy + nz z) times a
//               per-point factor folded in at packing
//   uoff        the point's own path-bin offset (laser leg of a non-confocal
//               scan, in bins; 0 for a confocal scan)
// An odd point count is padded with a point that never reaches a bin.
// ---------------------------------------------------------------------------
struct __align__(16) PointPair {
  float2 px, py, pz2, kq, na, nb, nc, uoff;
};
static_assert(sizeof(PointPair) == 64, "PointPair must be 64 bytes");

// Per-scan-point record: spot (sx, sy), bin offset off_s = (legs(s) - L0)/(c dt),
// and the transient's row in the caller's [scan_ny][scan_nx] layout. The
// forward reads its scan table in tile order (compact_tile_order), so that
// the 32 spots of a tile cover a compact 8 x 4 patch of the wall and its
// bounds rule out more (tile, point block) units.
struct __align__(16) ScanPoint {
  float sx, sy, off;
  uint32_t row;
};

// Scan points in tile order: 8 x 4 patches of the grid (x fastest), patches
// row by row; grids that are not multiples of the patch fill the last tiles
// of each patch row with the ragged remainder. out[k] = plain[order[k]].
void compact_tile_order(const std::vector<ScanPoint>& plain, uint32_t nx, uint32_t ny,
                        std::vector<ScanPoint>& out);

// Bounds of one sub-block of kSubPairs packed pairs (2 * kSubPairs points,
// in packed order), for the forward's unit culling:
//   x/y/z  box of the positions [m], n* box of the unit normals,
//   uo     range of the point's own path-bin offset (laser leg of a
//          non-confocal scan, in bins; 0 for confocal),
//   live   1 if some point can carry weight (albedo * area > 0 and, for a
//          non-confocal scan with object cosines, facing the laser), else 0.
constexpr uint32_t kSubPairs = 256;
struct __align__(16) BlockBound {
  float x0, x1, y0, y1, z0, z1;
  float nx0, nx1, ny0, ny1, nz0, nz1;
  float uo0, uo1, live, pad;
};
static_assert(sizeof(BlockBound) == 64, "BlockBound layout");

// Bounds of the scan spots of one tile of kTile scan points (valid ones):
// spot box and range of the bin offsets off_s.
struct __align__(16) TileBound {
  float sx0, sx1, sy0, sy1, off0, off1, pad0, pad1;
};
static_assert(sizeof(TileBound) == 32, "TileBound layout");

// Spatial order of the surface points: a counting sort by a 32^3 Morton cell
// of the scene's bounding box, so that a packed block holds nearby points
// and its bounds are tight.
constexpr uint32_t kOrderCells = 32768;

// Device scratch owned by a scene (one per scene). The error word is sticky
// (cleared by nlos_scene_check); the rest is reset by every forward pass.
struct SceneScratch {
  unsigned int err;           // kErr* bits
  unsigned int pad;
  // --- reset per pass from here ---
  unsigned int peak_bits;     // max of tau_G as float bits (values are >= 0)
  unsigned int pad2;
  unsigned long long boundary_pairs;
  double sum;                 // FP64 sum of tau_G over the cube
  double sumsq;               // FP64 sum of squares
  float scale;                // noise scale (computed on the device)
  float dark;
  unsigned long long pairs_full;  // pairs through the full evaluation (past the early out)
  unsigned long long next_chunk;  // forward: next chunk of work units to claim
  unsigned long long pairs_tested;  // pairs of the units the forward staged
  unsigned long long n_live;      // forward: entries of its live-unit list
};
constexpr size_t kScratchResetOffset = 8;  // offsetof(SceneScratch, peak_bits)
static_assert(sizeof(SceneScratch) == 80, "scratch layout");

struct Geometry {
  // host-side resolved parameters; a scene may hold scan rows [row0, row0 + ny)
  // of a grid of ny_full rows (a part of a cube split over devices)
  uint32_t nx, ny, B;
  uint32_t row0 = 0, ny_full = 0;
  uint64_t S, P;
  int scan_mode, cos_mode, bin_mode, noise_mode;
  double cdt;        // c * dt [m]
  double L0;         // window start [m]
  double sigma;      // jitter sigma in bins (0: none)
};

struct SceneImpl;

// Forward kernel launch (forward.cu). tau must be zeroed beforehand; the
// kernel adds its (jittered, for NEAREST) partial histograms into it.
cudaError_t launch_forward(const SceneImpl& sc, float* tau, cudaStream_t st);
cudaError_t launch_pair_table(const SceneImpl& sc, uint64_t s_begin, uint64_t s_count, float* u,
                              float* w, cudaStream_t st);
// Adjoint (backward.cu).
cudaError_t launch_backward(const SceneImpl& sc, const float* grad_tau, float* grad_albedo,
                            float* grad_depth, cudaStream_t st);

// Detector kernels (detector.cu).
int jitter_taps(double sigma, float* taps, int max_taps);  // returns k
cudaError_t launch_jitter(const float* in, float* out, uint64_t traces, uint32_t B, double sigma,
                          int replicate, cudaStream_t st);
// Replicate-padding correction weights of a jitter kernel: tail[k] = sum of the
// taps at offsets k + 1 .. R (k < R), i.e. the weight that output bin k (or
// B - 1 - k) draws from beyond the first (or last) bin.
void jitter_tails(const float* taps, int R, float* tail);
cudaError_t launch_reduce(const float* tau, uint64_t traces, uint32_t B, double* energy,
                          SceneScratch* scratch, cudaStream_t st);
// {max, sum, sum of squares} of a reduction's scratch as three doubles.
cudaError_t launch_stats_out(const SceneScratch* scratch, double* stats, cudaStream_t st);
cudaError_t launch_noise(const float* tau, uint64_t n, float scale, float dark, uint64_t seed,
                         uint32_t stream_tag, uint64_t index_base, uint32_t* counts,
                         cudaStream_t st);
// Noise for a scene: scale from the scene's reduction results (scratch), or,
// for a part of a larger cube, from the whole cube's {max, sum, sumsq}
// (cube_stats, device) over cube_bins bins; Philox streams of the global bin
// indices index_base + i.
cudaError_t launch_noise_scene(const float* tau, uint64_t n, SceneScratch* scratch, int mode,
                               float peak_photons, float dark, float nr_db, uint64_t seed,
                               uint32_t stream_tag, uint32_t* counts, cudaStream_t st,
                               uint64_t index_base = 0, const double* cube_stats = nullptr,
                               uint64_t cube_bins = 0);
cudaError_t launch_philox(const uint32_t* ctr, uint64_t n, uint32_t k0, uint32_t k1,
                          uint32_t* out, cudaStream_t st);

// Occluders of a scene (visibility extension): occ[2k] = (a.xyz, kind),
// occ[2k + 1] = (b.xyz, 0); kind 0 = sphere (centre a, radius b.x), 1 = box
// (corners a < b). Passed by value to the kernels that need it.
constexpr int kMaxOcc = NLOS_MAX_OCCLUDERS;
struct __align__(16) OccSet {
  int n;       // occluders in use (0: no visibility test)
  float eta;   // chord threshold, fraction of the segment
  float pad[2];
  float4 occ[2 * kMaxOcc];
};

// Scene internals shared by the host code of the library.
struct SceneImpl {
  nlos_params params;
  Geometry g;
  PointPair* pairs = nullptr;      // [ceil(P/2)] in spatial order
  ScanPoint* scan = nullptr;       // [S] in scan order (adjoint, pair table)
  ScanPoint* scan_fwd = nullptr;   // [S] in tile order (forward)
  SceneScratch* scratch = nullptr; // device
  float* raw_points = nullptr;     // [P][8] records the scene simulates (for the adjoint)
  float* base_points = nullptr;    // [P][8] records as given, once set_albedo_depth is used
  uint32_t* perm = nullptr;        // [P] packed position -> original point index
  uint16_t* cell = nullptr;        // [P] Morton cell of each point (ordering scratch)
  uint32_t* cells = nullptr;       // [kOrderCells + 8] counts/cursors + box (ordering scratch)
  BlockBound* bounds = nullptr;    // [ceil(P / 2 / kSubPairs)]
  TileBound* tiles = nullptr;      // [ceil(S / kTile)] of scan_fwd
  OccSet occ{};                    // occluders (host copy; n = 0: none)
  cudaStream_t stream = nullptr;   // creation stream
  int device = 0;
  int num_sms = 0;
};

int jitter_radius(double sigma);

// Spatial ordering, packing and block bounds of a scene's points (order.cu):
// the device counting sort, then the pack and bounds kernels, on stream st.
cudaError_t launch_order_pack(SceneImpl& s, cudaStream_t st);
// Tile bounds from a scan table (host).
void tile_bounds_host(const ScanPoint* sp, uint64_t S, std::vector<TileBound>& out);

}  // namespace nlos

struct nlos_scene {
  nlos::SceneImpl impl;
};
