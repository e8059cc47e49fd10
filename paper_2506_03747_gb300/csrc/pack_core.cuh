// Ingest/pack step of the GB300 NLOS simulator: per-point precomputation of
// the packed pair records (FP32 arithmetic, FP32 storage) with validation.
// Shared by scene creation and the persistent serving kernel.
#pragma once

#include "common.cuh"

namespace nlos {

// Part of the segment z -> x strictly inside occluder k of o, in units of the
// segment (FP64; the pack step's laser-leg visibility test).
__device__ inline double occ_chord64(const OccSet& o, int k, const double z[3],
                                     const double x[3]) {
  const float4 p = o.occ[2 * k], q = o.occ[2 * k + 1];
  const double d[3] = {x[0] - z[0], x[1] - z[1], x[2] - z[2]};
  double t0 = 0.0, t1 = 1.0;
  if (p.w == 0.f) {
    const double f[3] = {z[0] - (double)p.x, z[1] - (double)p.y, z[2] - (double)p.z};
    const double A = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double B = f[0] * d[0] + f[1] * d[1] + f[2] * d[2];
    const double C = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] - (double)q.x * (double)q.x;
    const double disc = B * B - A * C;
    if (!(A > 0.0) || !(disc > 0.0)) return 0.0;
    const double sq = sqrt(disc);
    t0 = fmax(t0, (-B - sq) / A);
    t1 = fmin(t1, (-B + sq) / A);
  } else {
    const double lo[3] = {p.x, p.y, p.z}, hi[3] = {q.x, q.y, q.z};
    for (int c = 0; c < 3; ++c) {
      if (d[c] == 0.0) {
        if (!(lo[c] < z[c] && z[c] < hi[c])) return 0.0;
        continue;
      }
      const double ta = (lo[c] - z[c]) / d[c], tb = (hi[c] - z[c]) / d[c];
      t0 = fmax(t0, fmin(ta, tb));
      t1 = fmin(t1, fmax(ta, tb));
    }
  }
  return t1 > t0 ? t1 - t0 : 0.0;
}

// Laser spot and 1 / (c dt) of the pack step as FP32 pairs (hi + lo carries
// the FP64 value to 48 bits), formed once on the host.
struct PackConst {
  float lx_hi, lx_lo, ly_hi, ly_lo, ic_hi, ic_lo;
};

inline PackConst pack_const(double lx, double ly, double inv_cdt) {
  PackConst c;
  c.lx_hi = (float)lx;
  c.lx_lo = (float)(lx - (double)c.lx_hi);
  c.ly_hi = (float)ly;
  c.ly_lo = (float)(ly - (double)c.ly_hi);
  c.ic_hi = (float)inv_cdt;
  c.ic_lo = (float)(inv_cdt - (double)c.ic_hi);
  return c;
}

// Laser leg l -> x of a non-confocal point, FP32: v = x - l, r_l = |v| and
// its offset r_l / (c dt) in bins. Each step rounds once (the square root is
// the correctly rounded one), so r_l is within ~1.5 ulp and the offset within
// ~2 ulp (1e-4 bin at 500 bins) of the FP64 values: far inside the bin-edge
// allowance of the forward, whose own FP32 path coordinate rounds at that level.
struct LaserLeg {
  float vx, vy, rl, uoff;
};

__device__ __forceinline__ LaserLeg laser_leg(float x, float y, float z, const PackConst& c) {
  LaserLeg g;
  g.vx = (x - c.lx_hi) - c.lx_lo;
  g.vy = (y - c.ly_hi) - c.ly_lo;
  g.rl = __fsqrt_rn(fmaf(g.vx, g.vx, fmaf(g.vy, g.vy, z * z)));
  g.uoff = fmaf(g.rl, c.ic_hi, g.rl * c.ic_lo);
  return g;
}

// Packs point pairs (FP32 arithmetic, correctly rounded steps; FP32 storage)
// and checks every point: finite values, z > 0, area > 0, albedo >= 0,
// |n| = 1 within 1e-3.
//   confocal:     OBJECT: (na, nb, nc) = -sqrt(q) * (nx, ny, nz z);
//                 WALL:   the same scaled by z; NONE: kq = q;
//   non-confocal: K = q * max(0, cos_l) / r_l^2 (laser leg l -> x),
//                 OBJECT: (na, nb, nc) = -K * (nx, ny, nz z); WALL: K * z / r_l * z;
//                 NONE: kq = q / r_l^2; uoff = r_l / (c dt).
// q = albedo * area. Every packed factor is within a few ulp of its FP64
// value (a relative error of a few 1e-7, against the 1e-6 energy bar).
// perm (nullable): packed position -> index of the point in raw.
// occ (nullable): occluders; non-confocal points hidden from the laser spot
// (a chord above occ->eta) get no weight (the chord test itself in FP64).
// The 8 values of one raw point (two 16-byte loads when the row is aligned).
__device__ __forceinline__ void load_point(const float* __restrict__ r, float v[8]) {
  if ((reinterpret_cast<uintptr_t>(r) & 15u) == 0) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(r));
    const float4 b = __ldg(reinterpret_cast<const float4*>(r) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
    for (int c = 0; c < 8; ++c) v[c] = __ldg(r + c);
  }
}

// rv (nullable): receives the raw values of the pair's points (the real ones).
__device__ __forceinline__ PointPair pack_pair_value(const float* __restrict__ raw, uint64_t P,
                                                     uint64_t k, int scan_mode, int cos_mode,
                                                     const PackConst& pc, unsigned int* err,
                                                     const uint32_t* __restrict__ perm,
                                                     const OccSet* occ = nullptr,
                                                     float (*rv)[8] = nullptr) {
  float f[2][8];
  for (int h = 0; h < 2; ++h) {
    const uint64_t i = 2 * k + h;
    if (i < P) {
      float r[8];
      load_point(raw + 8 * (perm ? (uint64_t)perm[i] : i), r);
      if (rv)
        for (int c = 0; c < 8; ++c) rv[h][c] = r[c];
      bool ok = true;
      for (int c = 0; c < 8; ++c) ok = ok && isfinite(r[c]);
      const float x = r[0], y = r[1], z = r[2], nx = r[3], ny = r[4], nz = r[5];
      // |n|^2 - 1 with one rounding of the sum of squares (a decision within
      // ~1e-7 of the 1e-3 threshold may differ from the FP64 one)
      const float nn = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
      ok = ok && z > 0.f && r[7] > 0.f && r[6] >= 0.f && fabsf(nn - 1.0f) <= 1e-3f;
      if (!ok) {
        atomicOr(err, kErrBadPoint);
      }
      const float q = r[6] * r[7];  // the FP64 product rounded once: the same float
      float kq = 0.f, s = 0.f, uoff = 0.f;
      if (scan_mode == NLOS_CONFOCAL) {
        if (cos_mode == NLOS_COS_NONE) kq = q;
        else if (cos_mode == NLOS_COS_OBJECT) s = __fsqrt_rn(q);
        else s = __fsqrt_rn(q) * z;
      } else {
        const LaserLeg g = laser_leg(x, y, z, pc);
        const float irl = __frcp_rn(g.rl);
        const float cl = -fmaf(nx, g.vx, fmaf(ny, g.vy, nz * z)) * irl;
        uoff = g.uoff;
        bool lit = true;
        if (occ) {
          const double zl[3] = {(double)pc.lx_hi + pc.lx_lo, (double)pc.ly_hi + pc.ly_lo, 0.0};
          const double xp[3] = {x, y, z};
          for (int k = 0; k < occ->n; ++k)
            if (occ_chord64(*occ, k, zl, xp) > (double)occ->eta) lit = false;
        }
        const float kl = q * irl * irl;
        if (!lit) {
          // no weight; kq = s = 0 below
        } else if (cos_mode == NLOS_COS_NONE) kq = kl;
        else if (cos_mode == NLOS_COS_OBJECT) s = kl * fmaxf(cl, 0.f);
        else s = kl * fmaxf(cl, 0.f) * (z * irl) * z;
      }
      f[h][0] = x;
      f[h][1] = y;
      f[h][2] = z * z;  // as the FP64 square rounded once
      f[h][3] = kq;
      f[h][4] = -s * nx;
      f[h][5] = -s * ny;
      f[h][6] = -s * (nz * z);
      f[h][7] = uoff;
    } else {
      // padding: far away, no weight, no cosine -> never binned
      f[h][0] = 0.f; f[h][1] = 0.f; f[h][2] = 1e30f; f[h][3] = 0.f;
      f[h][4] = 0.f; f[h][5] = 0.f; f[h][6] = 0.f; f[h][7] = 1e30f;
    }
  }
  PointPair o;
  o.px = make_float2(f[0][0], f[1][0]);
  o.py = make_float2(f[0][1], f[1][1]);
  o.pz2 = make_float2(f[0][2], f[1][2]);
  o.kq = make_float2(f[0][3], f[1][3]);
  o.na = make_float2(f[0][4], f[1][4]);
  o.nb = make_float2(f[0][5], f[1][5]);
  o.nc = make_float2(f[0][6], f[1][6]);
  o.uoff = make_float2(f[0][7], f[1][7]);
  return o;
}

__device__ __forceinline__ void pack_pair(const float* __restrict__ raw, uint64_t P, uint64_t k,
                                          int scan_mode, int cos_mode, const PackConst& pc,
                                          PointPair* pairs, unsigned int* err,
                                          const uint32_t* __restrict__ perm = nullptr,
                                          const OccSet* occ = nullptr) {
  pairs[k] = pack_pair_value(raw, P, k, scan_mode, cos_mode, pc, err, perm, occ);
}

// The per-point quantities of the block bounds: position, normal, laser-leg
// offset (non-confocal, the packed value), and whether the point can carry weight.
__device__ __forceinline__ void bound_point(const float* r, int scan_mode, int cos_mode,
                                            const PackConst& pc, float lo[7], float hi[7],
                                            float& live) {
  const float x = r[0], y = r[1], z = r[2];
  float uo = 0.f;
  bool w = r[6] * r[7] > 0.f;
  if (scan_mode == NLOS_NONCONFOCAL) {
    const LaserLeg g = laser_leg(x, y, z, pc);
    uo = g.uoff;
    if (cos_mode != NLOS_COS_NONE) w = w && -fmaf(r[3], g.vx, fmaf(r[4], g.vy, r[5] * z)) > 0.f;
  }
  const float v[7] = {x, y, z, r[3], r[4], r[5], uo};
  for (int c = 0; c < 7; ++c) {
    lo[c] = fminf(lo[c], v[c]);
    hi[c] = fmaxf(hi[c], v[c]);
  }
  if (w) live = 1.f;
}

__device__ __forceinline__ void bound_warp_reduce(float lo[7], float hi[7], float& live) {
  for (int o = 16; o > 0; o >>= 1) {
    for (int c = 0; c < 7; ++c) {
      lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
      hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
    }
    live = fmaxf(live, __shfl_xor_sync(0xffffffffu, live, o));
  }
}

__device__ __forceinline__ BlockBound bound_record(const float lo[7], const float hi[7],
                                                   float live) {
  BlockBound b;
  b.x0 = lo[0]; b.x1 = hi[0]; b.y0 = lo[1]; b.y1 = hi[1]; b.z0 = lo[2]; b.z1 = hi[2];
  b.nx0 = lo[3]; b.nx1 = hi[3]; b.ny0 = lo[4]; b.ny1 = hi[4]; b.nz0 = lo[5]; b.nz1 = hi[5];
  b.uo0 = lo[6]; b.uo1 = hi[6]; b.live = live; b.pad = 0.f;
  return b;
}

// Bounds of sub-block sb (points 2 kSubPairs sb .. in packed order) by one
// warp; lane 0 writes *out. Same per-point quantities as pack_pair.
__device__ __forceinline__ void block_bound_warp(const float* __restrict__ raw, uint64_t P,
                                                 uint64_t sb, int scan_mode, int cos_mode,
                                                 const PackConst& pc,
                                                 const uint32_t* __restrict__ perm,
                                                 BlockBound* out) {
  const int lane = threadIdx.x & 31;
  float lo[7], hi[7];
  for (int c = 0; c < 7; ++c) {
    lo[c] = 3.0e38f;
    hi[c] = -3.0e38f;
  }
  float live = 0.f;
  const uint64_t first = sb * 2 * kSubPairs;
  const uint64_t last = min(P, first + 2 * kSubPairs);
  for (uint64_t i = first + lane; i < last; i += 32)
    bound_point(raw + 8 * (perm ? (uint64_t)perm[i] : i), scan_mode, cos_mode, pc, lo, hi, live);
  bound_warp_reduce(lo, hi, live);
  if (lane == 0) *out = bound_record(lo, hi, live);
}

}  // namespace nlos
