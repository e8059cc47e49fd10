// Device steps of the spatial ordering of surface points (a counting sort by
// the Morton index of a 32 x 32 x 32 grid of cells over the points' bounding
// box), written as CTA-wide routines over a range of points so that both the
// standalone kernels (order.cu) and the persistent serving kernel (one range
// per work item) run them:
//   box_range      bounding box (order-preserving integer min/max atomics),
//   cell_range     each point's cell and the cell counts,
//   scan_cells     exclusive prefix sum of the counts (one CTA of 1024 threads),
//   scatter_range  perm[slot] = point, the slot from the cell's cursor.
#pragma once

#include "common.cuh"

namespace nlos {

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

// Words of the ordering scratch after the kOrderCells counts: min x, y, z and
// max x, y, z as ord_bits (initialised to all ones / zero), then padding.
constexpr uint32_t kOrderBoxWords = 8;

// Points [b, e), thread t0 of a grid-stride of `stride` threads; red: shared
// scratch of 6 words per warp of the CTA. All threads of the CTA call it.
__device__ __forceinline__ void box_range(const float* __restrict__ raw, uint64_t b, uint64_t e,
                                          uint64_t t0, uint64_t stride, uint32_t* box,
                                          uint32_t* red) {
  uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
  for (uint64_t i = b + t0; i < e; i += stride) {
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
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 3; ++c) {
      red[w * 6 + c] = mn[c];
      red[w * 6 + 3 + c] = mx[c];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int c = threadIdx.x;
    uint32_t v = red[c];
    for (int j = 1; j < (int)(blockDim.x >> 5); ++j)
      v = c < 3 ? min(v, red[j * 6 + c]) : max(v, red[j * 6 + c]);
    if (c < 3) atomicMin(&box[c], v);
    else atomicMax(&box[c], v);
  }
  __syncthreads();
}

__device__ __forceinline__ void cell_range(const float* __restrict__ raw, uint64_t b, uint64_t e,
                                           uint64_t t0, uint64_t stride, const uint32_t* box,
                                           uint16_t* cell, uint32_t* counts) {
  float lo[3], hi[3], inv[3];
  for (int c = 0; c < 3; ++c) {
    lo[c] = ord_float(box[c]);
    hi[c] = ord_float(box[3 + c]);
  }
  box_scale(lo, hi, inv);
  for (uint64_t i = b + t0; i < e; i += stride) {
    const uint32_t k = cell_of(raw[8 * i], raw[8 * i + 1], raw[8 * i + 2], lo, inv);
    cell[i] = (uint16_t)k;
    // one atomic per distinct cell of the warp: points given in grid or scan
    // order put a warp's 32 points in one or two cells, whose counter the
    // lanes would otherwise increment one after the other
    const unsigned peers = __match_any_sync(__activemask(), k);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&counts[k], (uint32_t)__popc(peers));
  }
}

// counts[c] <- sum of counts[0..c). One CTA of exactly 1024 threads: warp w
// scans cells [w * 1024, (w + 1) * 1024) 32 at a time (coalesced loads,
// shuffle scans), then the 32 warp totals are scanned; wsum: 32 shared words.
// PREFETCH loads a warp's 1024 counts into registers before the serial
// carry chain (32 loads in flight instead of one at a time; 32 registers).
template <bool PREFETCH = false>
__device__ __forceinline__ void scan_cells(uint32_t* counts, uint32_t* wsum) {
  constexpr int kPerWarp = kOrderCells / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* seg = counts + (size_t)w * kPerWarp;
  uint32_t pre[PREFETCH ? kPerWarp / 32 : 1];
  if (PREFETCH) {
#pragma unroll
    for (int j = 0; j < kPerWarp / 32; ++j) pre[j] = seg[32 * j + lane];
  }
  uint32_t carry = 0;
  auto step = [&](int j, uint32_t v) {
    uint32_t x = v;  // inclusive scan of the 32 values
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    seg[j + lane] = carry + x - v;  // exclusive within the warp's segment
    carry += __shfl_sync(0xffffffffu, x, 31);
  };
  if (PREFETCH) {
#pragma unroll
    for (int j = 0; j < kPerWarp; j += 32) step(j, pre[j / 32]);
  } else {
    for (int j = 0; j < kPerWarp; j += 32) step(j, seg[j + lane]);
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
  __syncthreads();
}

__device__ __forceinline__ void scatter_range(const uint16_t* cell, uint64_t b, uint64_t e,
                                              uint64_t t0, uint64_t stride, uint32_t* cursor,
                                              uint32_t* perm) {
  const uint32_t lane = threadIdx.x & 31;
  for (uint64_t i = b + t0; i < e; i += stride) {
    const uint32_t k = cell[i];
    // the lanes of one cell take consecutive slots from one atomic
    const unsigned peers = __match_any_sync(__activemask(), k);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if ((int)lane == leader) base = atomicAdd(&cursor[k], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    perm[base + (uint32_t)__popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

}  // namespace nlos
