// Spatial ordering of a scene's surface points, packing in that order, and
// the per-block bounds the forward kernel uses to skip (tile, block) units
// that cannot reach the acquisition window or face no spot of the tile.
//
// Ordering: a counting sort by the Morton index of a 32 x 32 x 32 grid of
// cells over the points' bounding box (cells in Z-order, points of a cell in
// arbitrary order), so that a packed block of 512 points covers a small part
// of the surface. The sum over points does not depend on the order; only the
// FP32 rounding of the histogram accumulation does.
//
// Device steps (one stream, no host synchronisation; the step routines are
// in order_core.cuh, shared with the serving kernel):
//   0. init: the cell counts zeroed, the box words set (one small kernel),
//   1. box: the points' bounding box (order-preserving integer atomics),
//   2. cell: each point's cell and the cell counts,
//   3. scan: exclusive prefix sum of the counts (one CTA),
//   4. scatter: perm[slot] = point, slot from the cell's cursor,
//   5. pack (pack_pair through perm) and block bounds, one CTA per sub-block.
#include "common.cuh"
#include "order_core.cuh"
#include "pack_core.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace nlos {

namespace {

__global__ void __launch_bounds__(256) box_kernel(const float* __restrict__ raw, uint64_t P,
                                                  uint32_t* box) {
  __shared__ uint32_t red[8 * 6];
  box_range(raw, 0, P, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
            (uint64_t)gridDim.x * blockDim.x, box, red);
}

__global__ void cell_kernel(const float* __restrict__ raw, uint64_t P, const uint32_t* box,
                            uint16_t* cell, uint32_t* counts) {
  cell_range(raw, 0, P, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
             (uint64_t)gridDim.x * blockDim.x, box, cell, counts);
}

// The cell counts zeroed and the box words set to their identities (min:
// all ones, max: zero) for the next ordering, in one launch.
__global__ void __launch_bounds__(256) order_init_kernel(uint32_t* counts, uint32_t* box) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  for (uint32_t i = t; i < kOrderCells; i += gridDim.x * blockDim.x) counts[i] = 0u;
  if (t < 6) box[t] = t < 3 ? 0xffffffffu : 0u;
}

__global__ void __launch_bounds__(1024) scan_kernel(uint32_t* counts) {
  __shared__ uint32_t wsum[32];
  scan_cells<true>(counts, wsum);
}

__global__ void scatter_kernel(const uint16_t* cell, uint64_t P, uint32_t* cursor, uint32_t* perm) {
  scatter_range(cell, 0, P, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                (uint64_t)gridDim.x * blockDim.x, cursor, perm);
}

// One CTA of kSubPairs threads per sub-block: thread k packs pair k of the
// sub-block, and the CTA reduces the bounds of its 2 kSubPairs points (the
// quantities of block_bound_warp, read off the packed record: the same
// laser-leg offsets, and liveness from the packed weight factor).
__global__ void __launch_bounds__(kSubPairs) pack_bounds_kernel(
    const float* __restrict__ raw, uint64_t P, int scan_mode, int cos_mode, const PackConst pc,
    const uint32_t* __restrict__ perm, PointPair* pairs, unsigned int* err,
    BlockBound* bounds, const __grid_constant__ OccSet occ) {
  static_assert(kSubPairs % 32 == 0 && kSubPairs <= 1024, "one thread per pair of a sub-block");
  __shared__ float red[kSubPairs / 32][15];
  const uint64_t n_pairs = (P + 1) / 2;
  const uint64_t k = (uint64_t)blockIdx.x * kSubPairs + threadIdx.x;
  // only the laser leg of a non-confocal scan is tested here
  const OccSet* o = (occ.n > 0 && scan_mode == NLOS_NONCONFOCAL) ? &occ : nullptr;
  float lo[7], hi[7], live = 0.f;
  for (int c = 0; c < 7; ++c) {
    lo[c] = 3.0e38f;
    hi[c] = -3.0e38f;
  }
  if (k < n_pairs) {
    float rv[2][8];
    const PointPair pp = pack_pair_value(raw, P, k, scan_mode, cos_mode, pc, err, perm, o, rv);
    pairs[k] = pp;
    // the bounds from the packed record and the raw values already loaded:
    // the laser-leg offset as packed, and "can carry weight" as a nonzero
    // packed weight factor (zero for albedo or area 0, a point facing away
    // from the laser, or one hidden from it)
    for (int h = 0; h < 2 && 2 * k + h < P; ++h) {
      const float* r = rv[h];
      const float kq = h ? pp.kq.y : pp.kq.x, na = h ? pp.na.y : pp.na.x;
      const float nb = h ? pp.nb.y : pp.nb.x, nc = h ? pp.nc.y : pp.nc.x;
      const float v[7] = {r[0], r[1], r[2], r[3], r[4], r[5], h ? pp.uoff.y : pp.uoff.x};
      for (int c = 0; c < 7; ++c) {
        lo[c] = fminf(lo[c], v[c]);
        hi[c] = fmaxf(hi[c], v[c]);
      }
      if (kq != 0.f || na != 0.f || nb != 0.f || nc != 0.f) live = 1.f;
    }
  }
  bound_warp_reduce(lo, hi, live);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    for (int c = 0; c < 7; ++c) {
      red[warp][c] = lo[c];
      red[warp][7 + c] = hi[c];
    }
    red[warp][14] = live;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kSubPairs / 32; ++w) {
      for (int c = 0; c < 7; ++c) {
        lo[c] = fminf(lo[c], red[w][c]);
        hi[c] = fmaxf(hi[c], red[w][7 + c]);
      }
      live = fmaxf(live, red[w][14]);
    }
    bounds[blockIdx.x] = bound_record(lo, hi, live);
  }
}

unsigned grid_for(uint64_t n, int per_block, int sms) {
  const uint64_t want = (n + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)sms * 8;
  return (unsigned)std::max<uint64_t>(1, std::min(want, cap));
}

}  // namespace

cudaError_t launch_order_pack(SceneImpl& s, cudaStream_t st) {
  const Geometry& g = s.g;
  const uint64_t P = g.P;
  if (P == 0) return cudaSuccess;
  uint32_t* counts = s.cells;
  uint32_t* box = s.cells + kOrderCells;
  order_init_kernel<<<32, 256, 0, st>>>(counts, box);
  box_kernel<<<grid_for(P, 2048, s.num_sms), 256, 0, st>>>(s.raw_points, P, box);
  cell_kernel<<<grid_for(P, 256, s.num_sms), 256, 0, st>>>(s.raw_points, P, box, s.cell, counts);
  scan_kernel<<<1, 1024, 0, st>>>(counts);
  scatter_kernel<<<grid_for(P, 256, s.num_sms), 256, 0, st>>>(s.cell, P, counts, s.perm);
  const uint64_t n_pairs = (P + 1) / 2;
  const PackConst pc = pack_const(s.params.laser_x, s.params.laser_y, 1.0 / g.cdt);
  const uint64_t n_sub = (n_pairs + kSubPairs - 1) / kSubPairs;
  pack_bounds_kernel<<<(unsigned)n_sub, kSubPairs, 0, st>>>(
      s.raw_points, P, g.scan_mode, g.cos_mode, pc, s.perm, s.pairs, &s.scratch->err,
      s.bounds, s.occ);
  return cudaGetLastError();
}

void tile_bounds_host(const ScanPoint* sp, uint64_t S, std::vector<TileBound>& out) {
  const uint64_t n = (S + kTile - 1) / kTile;
  out.assign(n, TileBound{});
  for (uint64_t t = 0; t < n; ++t) {
    TileBound b{3.0e38f, -3.0e38f, 3.0e38f, -3.0e38f, 3.0e38f, -3.0e38f, 0.f, 0.f};
    for (uint64_t s = t * kTile; s < std::min(S, (t + 1) * kTile); ++s) {
      b.sx0 = std::min(b.sx0, sp[s].sx);
      b.sx1 = std::max(b.sx1, sp[s].sx);
      b.sy0 = std::min(b.sy0, sp[s].sy);
      b.sy1 = std::max(b.sy1, sp[s].sy);
      b.off0 = std::min(b.off0, sp[s].off);
      b.off1 = std::max(b.off1, sp[s].off);
    }
    out[t] = b;
  }
}

}  // namespace nlos
