// Ingest/pack step of the GB300 NLOS simulator: per-point precomputation of
// the packed pair records (FP64 arithmetic, FP32 storage) with validation.
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

// Packs point pairs (FP64 arithmetic on the device, FP32 storage) and checks
// every point: finite values, z > 0, area > 0, albedo >= 0, |n| = 1 within 1e-3.
//   confocal:     OBJECT: (na, nb, nc) = -sqrt(q) * (nx, ny, nz z);
//                 WALL:   the same scaled by z; NONE: kq = q;
//   non-confocal: K = q * max(0, cos_l) / r_l^2 (laser leg l -> x),
//                 OBJECT: (na, nb, nc) = -K * (nx, ny, nz z); WALL: K * z / r_l * z;
//                 NONE: kq = q / r_l^2; uoff = r_l / (c dt).
// q = albedo * area.
// perm (nullable): packed position -> index of the point in raw.
// occ (nullable): occluders; non-confocal points hidden from the laser spot
// (a chord above occ->eta) get no weight.
__device__ __forceinline__ PointPair pack_pair_value(const float* __restrict__ raw, uint64_t P,
                                                     uint64_t k, int scan_mode, int cos_mode,
                                                     double lx, double ly, double inv_cdt,
                                                     unsigned int* err,
                                                     const uint32_t* __restrict__ perm,
                                                     const OccSet* occ = nullptr) {
  float f[2][8];
  for (int h = 0; h < 2; ++h) {
    const uint64_t i = 2 * k + h;
    if (i < P) {
      const float* r = raw + 8 * (perm ? (uint64_t)perm[i] : i);
      double nn = 0.0;
      bool ok = true;
      for (int c = 0; c < 8; ++c) ok = ok && isfinite(r[c]);
      nn = (double)r[3] * r[3] + (double)r[4] * r[4] + (double)r[5] * r[5];
      ok = ok && r[2] > 0.f && r[7] > 0.f && r[6] >= 0.f && fabs(nn - 1.0) <= 1e-3;
      if (!ok) {
        atomicOr(err, kErrBadPoint);
      }
      const double x = r[0], y = r[1], z = r[2], nx = r[3], ny = r[4], nz = r[5];
      const double q = (double)r[6] * (double)r[7];
      double kq = 0.0, s = 0.0, uoff = 0.0;
      if (scan_mode == NLOS_CONFOCAL) {
        if (cos_mode == NLOS_COS_NONE) kq = q;
        else if (cos_mode == NLOS_COS_OBJECT) s = sqrt(q);
        else s = sqrt(q) * z;
      } else {
        const double vx = x - lx, vy = y - ly, vz = z;
        const double rl = sqrt(vx * vx + vy * vy + vz * vz);
        const double irl = 1.0 / rl;  // one FP64 division (this part's FP64 pipe is slow)
        const double cl = -(nx * vx + ny * vy + nz * vz) * irl;
        uoff = rl * inv_cdt;
        bool lit = true;
        if (occ) {
          const double zl[3] = {lx, ly, 0.0}, xp[3] = {x, y, z};
          for (int k = 0; k < occ->n; ++k)
            if (occ_chord64(*occ, k, zl, xp) > (double)occ->eta) lit = false;
        }
        if (!lit) {
          // no weight; kq = s = 0 below
        } else if (cos_mode == NLOS_COS_NONE) kq = q * irl * irl;
        else if (cos_mode == NLOS_COS_OBJECT) s = q * (cl > 0 ? cl : 0.0) * irl * irl;
        else s = q * (cl > 0 ? cl : 0.0) * irl * irl * (z * irl) * z;
      }
      f[h][0] = (float)x;
      f[h][1] = (float)y;
      f[h][2] = (float)(z * z);
      f[h][3] = (float)kq;
      f[h][4] = (float)(-s * nx);
      f[h][5] = (float)(-s * ny);
      f[h][6] = (float)(-s * nz * z);
      f[h][7] = (float)uoff;
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
                                          int scan_mode, int cos_mode, double lx, double ly,
                                          double inv_cdt, PointPair* pairs, unsigned int* err,
                                          const uint32_t* __restrict__ perm = nullptr,
                                          const OccSet* occ = nullptr) {
  pairs[k] = pack_pair_value(raw, P, k, scan_mode, cos_mode, lx, ly, inv_cdt, err, perm, occ);
}

// The per-point quantities of the block bounds: position, normal, laser-leg
// offset (non-confocal), and whether the point can carry weight.
__device__ __forceinline__ void bound_point(const float* r, int scan_mode, int cos_mode, double lx,
                                            double ly, double inv_cdt, float lo[7], float hi[7],
                                            float& live) {
  const float x = r[0], y = r[1], z = r[2];
  float uo = 0.f;
  bool w = r[6] * r[7] > 0.f;
  if (scan_mode == NLOS_NONCONFOCAL) {
    const double vx = x - lx, vy = y - ly, vz = z;
    const double rl = sqrt(vx * vx + vy * vy + vz * vz);
    uo = (float)(rl * inv_cdt);
    if (cos_mode != NLOS_COS_NONE) w = w && -(r[3] * vx + r[4] * vy + r[5] * vz) > 0.0;
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
                                                 double lx, double ly, double inv_cdt,
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
    bound_point(raw + 8 * (perm ? (uint64_t)perm[i] : i), scan_mode, cos_mode, lx, ly, inv_cdt,
                lo, hi, live);
  bound_warp_reduce(lo, hi, live);
  if (lane == 0) *out = bound_record(lo, hi, live);
}

}  // namespace nlos
