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
// Device steps (one stream, no host synchronisation):
//   1. box: the points' bounding box (order-preserving integer atomics),
//   2. cell: each point's cell and the cell counts,
//   3. scan: exclusive prefix sum of the counts (one CTA),
//   4. scatter: perm[slot] = point, slot from the cell's cursor,
//   5. pack (pack_pair through perm) and block bounds (one warp per block).
#include "common.cuh"
#include "pack_core.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace nlos {

namespace {


// float -> unsigned with the same order
__host__ __device__ inline uint32_t ord_bits(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ inline float ord_float(uint32_t u) {
  const uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  float f;
  memcpy(&f, &b, 4);
  return f;
}

__host__ __device__ inline uint32_t spread5(uint32_t v) {
  uint32_t o = 0;
  for (int b = 0; b < 5; ++b) o |= ((v >> b) & 1u) << (3 * b);
  return o;
}

__host__ __device__ inline uint32_t cell_of(float x, float y, float z, const float* lo,
                                            const float* inv) {
  const float v[3] = {x, y, z};
  uint32_t q[3];
  for (int c = 0; c < 3; ++c) {
    const float t = (v[c] - lo[c]) * inv[c];
    q[c] = t > 0.f ? (uint32_t)fminf(t, 31.f) : 0u;
  }
  return spread5(q[0]) | (spread5(q[1]) << 1) | (spread5(q[2]) << 2);
}

__host__ __device__ inline void box_scale(const float* lo, const float* hi, float* inv) {
  for (int c = 0; c < 3; ++c) {
    const float ext = hi[c] - lo[c];
    inv[c] = ext > 0.f ? 32.0f / ext : 0.f;
  }
}

__global__ void __launch_bounds__(256) box_kernel(const float* __restrict__ raw, uint64_t P,
                                                  uint32_t* box) {
  uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (uint64_t)gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const uint32_t u = ord_bits(raw[8 * i + c]);
      mn[c] = min(mn[c], u);
      mx[c] = max(mx[c], u);
    }
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int c = 0; c < 3; ++c) {
      mn[c] = min(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
      mx[c] = max(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
    }
  // CTA reduction first: one global atomic per CTA and word (same-address
  // atomics from every warp serialise)
  __shared__ uint32_t s[8][6];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 3; ++c) {
      s[w][c] = mn[c];
      s[w][3 + c] = mx[c];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int c = threadIdx.x;
    uint32_t v = s[0][c];
    for (int j = 1; j < (int)(blockDim.x >> 5); ++j) v = c < 3 ? min(v, s[j][c]) : max(v, s[j][c]);
    if (c < 3) atomicMin(&box[c], v);
    else atomicMax(&box[c], v);
  }
}

__global__ void cell_kernel(const float* __restrict__ raw, uint64_t P, const uint32_t* box,
                            uint16_t* cell, uint32_t* counts) {
  float lo[3], hi[3], inv[3];
  for (int c = 0; c < 3; ++c) {
    lo[c] = ord_float(box[c]);
    hi[c] = ord_float(box[3 + c]);
  }
  box_scale(lo, hi, inv);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t k = cell_of(raw[8 * i], raw[8 * i + 1], raw[8 * i + 2], lo, inv);
    cell[i] = (uint16_t)k;
    atomicAdd(&counts[k], 1u);
  }
}

// One CTA of 1024 threads: counts[c] <- sum of counts[0..c). Warp w scans
// cells [w * 1024, (w + 1) * 1024) 32 at a time (coalesced loads, shuffle
// scans), then the 32 warp totals are scanned.
__global__ void __launch_bounds__(1024) scan_kernel(uint32_t* counts) {
  constexpr int kPerWarp = kOrderCells / 32;
  __shared__ uint32_t wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* seg = counts + (size_t)w * kPerWarp;
  uint32_t carry = 0;
  for (int j = 0; j < kPerWarp; j += 32) {
    const uint32_t v = seg[j + lane];
    uint32_t x = v;  // inclusive scan of the 32 values
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    seg[j + lane] = carry + x - v;  // exclusive within the warp's segment
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) wsum[w] = carry;
  __syncthreads();
  if (w == 0) {
    const uint32_t v = wsum[lane];
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    wsum[lane] = x - v;
  }
  __syncthreads();
  const uint32_t base = wsum[w];
  for (int j = lane; j < kPerWarp; j += 32) seg[j] += base;
}

__global__ void scatter_kernel(const uint16_t* cell, uint64_t P, uint32_t* cursor, uint32_t* perm) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (uint64_t)gridDim.x * blockDim.x)
    perm[atomicAdd(&cursor[cell[i]], 1u)] = (uint32_t)i;
}

__global__ void pack_perm_kernel(const float* __restrict__ raw, uint64_t P, int scan_mode,
                                 int cos_mode, double lx, double ly, double inv_cdt,
                                 const uint32_t* __restrict__ perm, PointPair* pairs,
                                 unsigned int* err) {
  const uint64_t n_pairs = (P + 1) / 2;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_pairs;
       k += (uint64_t)gridDim.x * blockDim.x)
    pack_pair(raw, P, k, scan_mode, cos_mode, lx, ly, inv_cdt, pairs, err, perm);
}

__global__ void bounds_kernel(const float* __restrict__ raw, uint64_t P, int scan_mode,
                              int cos_mode, double lx, double ly, double inv_cdt,
                              const uint32_t* __restrict__ perm, BlockBound* bounds,
                              uint64_t n_sub) {
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t sb = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sb < n_sub;
       sb += warps)
    block_bound_warp(raw, P, sb, scan_mode, cos_mode, lx, ly, inv_cdt, perm, bounds + sb);
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
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * kOrderCells, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(box, 0xff, sizeof(uint32_t) * 3, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(box + 3, 0, sizeof(uint32_t) * 3, st);
  if (e != cudaSuccess) return e;
  box_kernel<<<grid_for(P, 2048, s.num_sms), 256, 0, st>>>(s.raw_points, P, box);
  cell_kernel<<<grid_for(P, 256, s.num_sms), 256, 0, st>>>(s.raw_points, P, box, s.cell, counts);
  scan_kernel<<<1, 1024, 0, st>>>(counts);
  scatter_kernel<<<grid_for(P, 256, s.num_sms), 256, 0, st>>>(s.cell, P, counts, s.perm);
  const uint64_t n_pairs = (P + 1) / 2;
  const double lx = s.params.laser_x, ly = s.params.laser_y, inv_cdt = 1.0 / g.cdt;
  pack_perm_kernel<<<grid_for(n_pairs, 256, s.num_sms), 256, 0, st>>>(
      s.raw_points, P, g.scan_mode, g.cos_mode, lx, ly, inv_cdt, s.perm, s.pairs, &s.scratch->err);
  const uint64_t n_sub = (n_pairs + kSubPairs - 1) / kSubPairs;
  bounds_kernel<<<grid_for(n_sub, 8, s.num_sms), 256, 0, st>>>(
      s.raw_points, P, g.scan_mode, g.cos_mode, lx, ly, inv_cdt, s.perm, s.bounds, n_sub);
  return cudaGetLastError();
}

void order_points_host(const float* pts, uint64_t P, float* out) {
  if (P == 0) return;
  float lo[3], hi[3], inv[3];
  for (int c = 0; c < 3; ++c) lo[c] = hi[c] = pts[c];
  for (uint64_t i = 1; i < P; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], pts[8 * i + c]);
      hi[c] = std::max(hi[c], pts[8 * i + c]);
    }
  box_scale(lo, hi, inv);
  std::vector<uint32_t> start(kOrderCells + 1, 0);
  std::vector<uint16_t> cell(P);
  for (uint64_t i = 0; i < P; ++i) {
    cell[i] = (uint16_t)cell_of(pts[8 * i], pts[8 * i + 1], pts[8 * i + 2], lo, inv);
    ++start[cell[i] + 1];
  }
  for (uint32_t c = 0; c < kOrderCells; ++c) start[c + 1] += start[c];
  for (uint64_t i = 0; i < P; ++i) {
    const uint32_t slot = start[cell[i]]++;
    std::copy(pts + 8 * i, pts + 8 * i + 8, out + 8 * (uint64_t)slot);
  }
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
