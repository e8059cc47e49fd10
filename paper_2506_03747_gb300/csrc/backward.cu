// Adjoint of the Gaussian-splat forward (differentiable form of the binned
// transient of arXiv 2506.03747): gradients of a loss L(tau) with respect to
// per-point albedo rho_p and per-point displacement delta_p along the normal.
//
// For a pair (s, p) with x_b = b + 1/2 - u_sp and phi the splat kernel,
//   G0 = sum_b g[s][b] phi(x_b),   G1 = sum_b g[s][b] (x_b / sigma^2) phi(x_b),
//   dL/d rho_p   = sum_s (dw/d rho) G0,
//   dL/d delta_p = sum_s (dw/d delta) G0 + w (du/d delta) G1,
// with, for x -> x + delta n: dr/d delta = -cos, d cos/d delta = -(1 - cos^2)/r,
// d(z/r)/d delta = (n_z + (z/r) cos)/r and du/d delta = -(cos_l + cos_d)/(c dt).
//
// Two forms of the sums G0, G1:
//  * taps (any sigma): one CTA per (32-scan-point tile, point block); the
//    tile's g rows are staged into shared memory as [bin][32] (lane = scan
//    point, conflict-free gathers) and each lane runs the |x_b| < 6 sigma taps
//    of its own pair;
//  * moments (sigma >= 2.5 bins): with u = j + f (j = floor u), c = 1/2 - f
//    and m = b - j, x_b = m + c, and the Taylor expansion
//    phi(m + c) = sum_{n < N} D_n[m] c^n (the table of the moment forward)
//    turns the sums into polynomials in c,
//      G0 = sum_n c^n H_n[j],                   H_n[j] = sum_m g[j + m] D_n[m],
//      sigma^2 G1 = sum_n c^n M_n[j] + c G0,    M_n[j] = sum_m g[j + m] m D_n[m],
//    so a first kernel correlates every transient of g with the 2N tables
//    (2N floats per (s, j)) and the pair kernel needs one 48-byte gather and
//    two Horner evaluations per pair instead of about 12 sigma taps.
// Taps form: points are broadcast from shared memory, and a warp sum over the
// 32 scan points of a tile gives the tile's contribution to each point, added
// to the outputs with one global atomic. Moments form: one thread per point,
// looping over a block of scan points broadcast from shared memory; the sums
// over s stay in the thread's registers (no warp sum), the laser leg of a
// non-confocal scan is computed once per point, and each block of scan points
// adds its contribution to each point with one global atomic.
#include "common.cuh"
#include "device_util.cuh"
#include "forward_core.cuh"

#include <cmath>

namespace nlos {

namespace {

constexpr int kBwdTile = 32;
constexpr int kBwdPoints = 256;  // points per CTA
constexpr int kBwdMomThreads = 256;  // moments form: points per CTA (one per thread)
constexpr int kBwdMomScan = 128;     // moments form: scan points per CTA
constexpr int kAdjTabThreads = 256;
static_assert(kMoments == 6, "the adjoint table holds 2 x 6 moments in three float4");

struct BwdArgs {
  const float* raw;        // [P][8]
  const ScanPoint* scan;   // spots and offsets
  const float* g;          // [S][B]
  float* ga;               // [P] or null
  float* gd;               // [P] or null
  uint64_t P, S;
  uint32_t B;
  int scan_mode, cos_mode;
  float lx, ly;            // laser spot (non-confocal)
  float inv_cdt;           // 1 / (c dt)
  float inv2s2, inv_s2, norm, reach, qstep;
};

#ifndef NLOS_BWD_RSQRT
#define NLOS_BWD_RSQRT 1  // legs from a reciprocal square root estimate and one Newton step
#endif

// 1 / sqrt(x) for x > 0: the hardware estimate and one Newton step (about an
// ulp; the gradients are held to 1e-3 of their maximum).
__device__ __forceinline__ float rsqrt_newton(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y * fmaf(-0.5f * x, y * y, 1.5f);
}

// A leg's length and its reciprocal from its squared length.
__device__ __forceinline__ void leg_length(float r2, float& r, float& ri) {
#if NLOS_BWD_RSQRT
  ri = rsqrt_newton(r2);
  r = r2 * ri;
#else
  r = sqrtf(r2);
  ri = 1.0f / r;
#endif
}

// Leg factor F = cosf * wallf / r^2 and its delta-derivative (FP32); ri = 1 / r.
__device__ __forceinline__ void leg(int cos_mode, float ndotv, float vz, float nz, float ri,
                                    float& F, float& dF, float& c) {
  c = -ndotv * ri;
  const float dc = -(1.0f - c * c) * ri;
  float fc = 1.0f, dfc = 0.0f;
  if (cos_mode >= NLOS_COS_OBJECT) {
    if (c > 0.0f) {
      fc = c;
      dfc = dc;
    } else {
      fc = 0.0f;
      dfc = 0.0f;
    }
  }
  float fw = 1.0f, dfw = 0.0f;
  if (cos_mode == NLOS_COS_OBJECT_WALL) {
    fw = vz * ri;
    dfw = (nz + fw * c) * ri;
  }
  const float ri2 = ri * ri;
  F = fc * fw * ri2;
  // d(r^-2)/d delta = -2 r^-3 dr/d delta = 2 c r^-3
  dF = (dfc * fw + fc * dfw) * ri2 + fc * fw * 2.0f * c * ri2 * ri;
}

// H_n[j], M_n[j] of one transient for j = r - J, r in [0, rows), rows = B + 2J,
// as T[s][r] = {H_0..H_3}, {H_4, H_5, M_0, M_1}, {M_2..M_5}.
struct AdjTabArgs {
  const float* g;  // [S][B]
  float4* T;       // [S][rows][3]
  uint64_t S;
  uint32_t B, rows, row_blocks;
};

__global__ void __launch_bounds__(kAdjTabThreads)
    adj_table_kernel(const AdjTabArgs a, const __grid_constant__ MomTab mt) {
  __shared__ float gs[kAdjTabThreads + 2 * kMomMaxJ];
  const uint64_t s = blockIdx.x / a.row_blocks;
  const int r0 = (int)(blockIdx.x % a.row_blocks) * kAdjTabThreads;
  const int J = mt.J;
  // gs[i] = g[s][r0 - 2J + i] (zero outside the transient)
  for (int i = threadIdx.x; i < kAdjTabThreads + 2 * J; i += blockDim.x) {
    const int b = r0 - 2 * J + i;
    gs[i] = (b >= 0 && b < (int)a.B) ? a.g[s * a.B + b] : 0.0f;
  }
  __syncthreads();
  const int r = r0 + (int)threadIdx.x;
  if (r >= (int)a.rows) return;
  float h[kMoments], mm[kMoments];
#pragma unroll
  for (int n = 0; n < kMoments; ++n) h[n] = mm[n] = 0.0f;
  // g[j + m] with j = r - J is gs[threadIdx.x + J + m]
  const float* gp = gs + threadIdx.x + J;
  for (int m = -J; m <= J; ++m) {
    const float gv = gp[m];
    const float gm = gv * (float)m;
#pragma unroll
    for (int n = 0; n < kMoments; ++n) {
      const float d = mt.d[n][m + J];
      h[n] = fmaf(gv, d, h[n]);
      mm[n] = fmaf(gm, d, mm[n]);
    }
  }
  float4* out = a.T + (s * a.rows + (uint64_t)r) * 3;
  out[0] = make_float4(h[0], h[1], h[2], h[3]);
  out[1] = make_float4(h[4], h[5], mm[0], mm[1]);
  out[2] = make_float4(mm[2], mm[3], mm[4], mm[5]);
}

__device__ __forceinline__ float horner6(float c, float p0, float p1, float p2, float p3, float p4,
                                         float p5) {
  return fmaf(fmaf(fmaf(fmaf(fmaf(p5, c, p4), c, p3), c, p2), c, p1), c, p0);
}

// Taps form: one CTA per (32-scan-point tile, block of kBwdPoints points).
__global__ void __launch_bounds__(256) bwd_kernel(const BwdArgs a) {
  extern __shared__ float sm[];
  float* gt = sm;                              // [B][32]
  float* pts = sm + (size_t)a.B * kBwdTile;    // [kBwdPoints][8]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const uint64_t n_pblk = (a.P + kBwdPoints - 1) / kBwdPoints;
  const uint64_t tile = blockIdx.x / n_pblk;
  const uint64_t p0 = (blockIdx.x % n_pblk) * kBwdPoints;
  const int np = (int)min((uint64_t)kBwdPoints, a.P - p0);

  for (uint32_t i = tid; i < a.B * kBwdTile; i += blockDim.x) {
    const uint32_t s_loc = i & 31, b = i >> 5;
    const uint64_t s = tile * kBwdTile + s_loc;
    gt[i] = s < a.S ? a.g[s * a.B + b] : 0.0f;
  }
  for (int i = tid; i < np * 8; i += blockDim.x) pts[i] = a.raw[p0 * 8 + i];
  __syncthreads();

  const uint64_t s = tile * kBwdTile + lane;
  const bool valid = s < a.S;
  ScanPoint sp = valid ? a.scan[s] : ScanPoint{0.f, 0.f, -1e30f, 0u};
  const float dx_s = sp.sx, dy_s = sp.sy;
  const float lx = a.scan_mode == NLOS_CONFOCAL ? sp.sx : a.lx;
  const float ly = a.scan_mode == NLOS_CONFOCAL ? sp.sy : a.ly;

  for (int i = warp; i < np; i += nwarps) {
    const float* q = pts + 8 * i;
    const float x = q[0], y = q[1], z = q[2], nx = q[3], ny = q[4], nz = q[5], rho = q[6],
                area = q[7];
    // laser leg l -> x and detector leg d -> x
    const float vlx = x - lx, vly = y - ly, vlz = z;
    float rl, ril;
    leg_length(vlx * vlx + vly * vly + vlz * vlz, rl, ril);
    float Fl, dFl, cl, Fd, dFd, cd, rd;
    leg(a.cos_mode, nx * vlx + ny * vly + nz * vlz, vlz, nz, ril, Fl, dFl, cl);
    if (a.scan_mode == NLOS_CONFOCAL) {
      // the laser spot is the detector spot: the second leg is the first
      rd = rl;
      Fd = Fl;
      dFd = dFl;
      cd = cl;
    } else {
      const float vdx = x - dx_s, vdy = y - dy_s, vdz = z;
      float rid;
      leg_length(vdx * vdx + vdy * vdy + vdz * vdz, rd, rid);
      leg(a.cos_mode, nx * vdx + ny * vdy + nz * vdz, vdz, nz, rid, Fd, dFd, cd);
    }
    const float qw = rho * area;
    const float w = qw * Fl * Fd;
    const float dw_drho = area * Fl * Fd;
    const float dw_dd = qw * (dFl * Fd + Fl * dFd);
    // u relative to bin 0: legs and window start are in sp.off (both legs
    // below are recomputed here rather than taken from the packed form)
    const float u = (rl + rd) * a.inv_cdt + sp.off;
    const float du_dd = -(cl + cd) * a.inv_cdt;
    float G0 = 0.f, G1 = 0.f;
    if (valid && (w != 0.f || dw_dd != 0.f || dw_drho != 0.f)) {
      const int lo = max(0, (int)(floorf(u - 0.5f - a.reach) + 1.0f));
      const int hi = min((int)a.B - 1, (int)(ceilf(u - 0.5f + a.reach) - 1.0f));
      if (lo <= hi) {
        // tap recurrence restarted every 8 taps (its rounding error grows
        // with the square of the number of steps)
        float K = 0.f, r = 0.f;
        for (int b = lo; b <= hi; ++b) {
          const float xb = (float)b + 0.5f - u;
          if (((b - lo) & 7) == 0) {
            K = a.norm * expf(-xb * xb * a.inv2s2);
            r = expf(-(2.0f * xb + 1.0f) * a.inv2s2);
          }
          const float gv = gt[b * kBwdTile + lane];
          G0 = fmaf(gv, K, G0);
          G1 = fmaf(gv * xb, K, G1);
          K *= r;
          r *= a.qstep;
        }
        G1 *= a.inv_s2;
      }
    }
    float ca = dw_drho * G0;
    float cdl = dw_dd * G0 + w * du_dd * G1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ca += __shfl_xor_sync(0xffffffffu, ca, o);
      cdl += __shfl_xor_sync(0xffffffffu, cdl, o);
    }
    if (lane == 0) {
      if (a.ga) atomicAdd(a.ga + p0 + i, ca);
      if (a.gd) atomicAdd(a.gd + p0 + i, cdl);
    }
  }
}

// Moments form: thread = point p0 + threadIdx.x, CTA = (block of scan points,
// block of points) with the scan block the slower index, so the CTAs resident
// at one time read the moment tables of few transients. T[s][r] as written by
// adj_table_kernel, rows = B + 2J.
template <int SCAN, int COS>
__global__ void __launch_bounds__(kBwdMomThreads)
    bwd_mom_kernel(const BwdArgs a, const float4* __restrict__ T, int J, uint32_t rows,
                   uint32_t n_pblk) {
  __shared__ ScanPoint ss[kBwdMomScan];
  const uint64_t s0 = (uint64_t)(blockIdx.x / n_pblk) * kBwdMomScan;
  const uint64_t p = (uint64_t)(blockIdx.x % n_pblk) * kBwdMomThreads + threadIdx.x;
  const int ns = (int)min((uint64_t)kBwdMomScan, a.S - s0);
  for (int i = threadIdx.x; i < ns; i += blockDim.x) ss[i] = a.scan[s0 + i];
  __syncthreads();
  if (p >= a.P) return;
  const float4* rp = reinterpret_cast<const float4*>(a.raw + p * 8);
  const float4 q0 = rp[0], q1 = rp[1];
  const float x = q0.x, y = q0.y, z = q0.z, nx = q0.w, ny = q1.x, nz = q1.y, rho = q1.z,
              area = q1.w;
  const float z2 = z * z, nzz = nz * z, qw = rho * area;
  // the laser leg of a non-confocal scan depends on the point only
  float rl = 0.f, Fl = 0.f, dFl = 0.f, cl = 0.f;
  if (SCAN != NLOS_CONFOCAL) {
    const float vlx = x - a.lx, vly = y - a.ly;
    float ril;
    leg_length(fmaf(vlx, vlx, fmaf(vly, vly, z2)), rl, ril);
    leg(COS, fmaf(nx, vlx, fmaf(ny, vly, nzz)), z, nz, ril, Fl, dFl, cl);
  }
  const float rows_hi = (float)((int)rows - J);
  float ca = 0.f, cdl = 0.f;
  for (int k = 0; k < ns; ++k) {
    const ScanPoint sp = ss[k];
    // the detector leg d -> x (for a confocal scan also the laser leg)
    const float vdx = x - sp.sx, vdy = y - sp.sy;
    float rd, rid, Fd, dFd, cd;
    leg_length(fmaf(vdx, vdx, fmaf(vdy, vdy, z2)), rd, rid);
    leg(COS, fmaf(nx, vdx, fmaf(ny, vdy, nzz)), z, nz, rid, Fd, dFd, cd);
    float w, dw_drho, dw_dd, u, du_dd;
    if (SCAN == NLOS_CONFOCAL) {
      const float F2 = Fd * Fd;
      w = qw * F2;
      dw_drho = area * F2;
      dw_dd = qw * 2.0f * Fd * dFd;
      u = 2.0f * rd * a.inv_cdt + sp.off;
      du_dd = -2.0f * cd * a.inv_cdt;
    } else {
      const float F2 = Fl * Fd;
      w = qw * F2;
      dw_drho = area * F2;
      dw_dd = qw * (dFl * Fd + Fl * dFd);
      u = (rl + rd) * a.inv_cdt + sp.off;
      du_dd = -(cl + cd) * a.inv_cdt;
    }
    const float fl = floorf(u);
    if ((w != 0.f || dw_dd != 0.f || dw_drho != 0.f) && fl >= (float)-J && fl < rows_hi) {
      const float c = 0.5f - (u - fl);
      const float4* t = T + ((s0 + (uint64_t)k) * rows + (uint64_t)((int)fl + J)) * 3;
      const float4 t0 = __ldg(t), t1 = __ldg(t + 1), t2 = __ldg(t + 2);
      const float G0 = horner6(c, t0.x, t0.y, t0.z, t0.w, t1.x, t1.y);
      const float gm = horner6(c, t1.z, t1.w, t2.x, t2.y, t2.z, t2.w);
      const float G1 = fmaf(c, G0, gm) * a.inv_s2;
      ca = fmaf(dw_drho, G0, ca);
      cdl = fmaf(dw_dd, G0, fmaf(w * du_dd, G1, cdl));
    }
  }
  if (a.ga) atomicAdd(a.ga + p, ca);
  if (a.gd) atomicAdd(a.gd + p, cdl);
}

using BwdMomFn = void (*)(const BwdArgs, const float4*, int, uint32_t, uint32_t);

BwdMomFn pick_mom(int scan_mode, int cos_mode) {
  if (scan_mode == NLOS_CONFOCAL) {
    if (cos_mode == NLOS_COS_NONE) return bwd_mom_kernel<NLOS_CONFOCAL, NLOS_COS_NONE>;
    if (cos_mode == NLOS_COS_OBJECT) return bwd_mom_kernel<NLOS_CONFOCAL, NLOS_COS_OBJECT>;
    return bwd_mom_kernel<NLOS_CONFOCAL, NLOS_COS_OBJECT_WALL>;
  }
  if (cos_mode == NLOS_COS_NONE) return bwd_mom_kernel<NLOS_NONCONFOCAL, NLOS_COS_NONE>;
  if (cos_mode == NLOS_COS_OBJECT) return bwd_mom_kernel<NLOS_NONCONFOCAL, NLOS_COS_OBJECT>;
  return bwd_mom_kernel<NLOS_NONCONFOCAL, NLOS_COS_OBJECT_WALL>;
}

}  // namespace

cudaError_t launch_backward(const SceneImpl& sc, const float* grad_tau, float* grad_albedo,
                            float* grad_depth, cudaStream_t st) {
  const Geometry& g = sc.g;
  cudaError_t e;
  if (grad_albedo && (e = cudaMemsetAsync(grad_albedo, 0, sizeof(float) * g.P, st)) != cudaSuccess)
    return e;
  if (grad_depth && (e = cudaMemsetAsync(grad_depth, 0, sizeof(float) * g.P, st)) != cudaSuccess)
    return e;
  if (g.P == 0 || g.S == 0) return cudaSuccess;
  BwdArgs a{};
  a.raw = sc.raw_points;
  a.scan = sc.scan;
  a.g = grad_tau;
  a.ga = grad_albedo;
  a.gd = grad_depth;
  a.P = g.P;
  a.S = g.S;
  a.B = g.B;
  a.scan_mode = g.scan_mode;
  a.cos_mode = g.cos_mode;
  a.lx = (float)sc.params.laser_x;
  a.ly = (float)sc.params.laser_y;
  a.inv_cdt = (float)(1.0 / g.cdt);
  const double s = g.sigma;
  a.inv2s2 = (float)(1.0 / (2.0 * s * s));
  a.inv_s2 = (float)(1.0 / (s * s));
  a.norm = (float)(1.0 / (s * std::sqrt(2.0 * 3.14159265358979323846)));
  a.reach = (float)(6.0 * s);
  a.qstep = (float)std::exp(-1.0 / (s * s));
  if (use_moments(s)) {
    // moment tables: S x (B + 2J) x 48 bytes, stream-ordered, freed after use
    MomTab mt;
    moment_table(s, mt);
    AdjTabArgs t{};
    t.g = grad_tau;
    t.S = g.S;
    t.B = g.B;
    t.rows = g.B + 2u * (uint32_t)mt.J;
    t.row_blocks = (t.rows + kAdjTabThreads - 1) / kAdjTabThreads;
    const uint64_t tab_blocks = g.S * t.row_blocks;
    if (tab_blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    e = cudaMallocAsync(reinterpret_cast<void**>(&t.T), sizeof(float4) * 3 * g.S * t.rows, st);
    if (e != cudaSuccess) return e;
    adj_table_kernel<<<(unsigned)tab_blocks, kAdjTabThreads, 0, st>>>(t, mt);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      const uint64_t n_pblk = (g.P + kBwdMomThreads - 1) / kBwdMomThreads;
      const uint64_t mblocks = n_pblk * ((g.S + kBwdMomScan - 1) / kBwdMomScan);
      if (mblocks > 0x7fffffffull) {
        e = cudaErrorInvalidValue;
      } else {
        pick_mom(g.scan_mode, g.cos_mode)<<<(unsigned)mblocks, kBwdMomThreads, 0, st>>>(
            a, t.T, mt.J, t.rows, (uint32_t)n_pblk);
        e = cudaGetLastError();
      }
    }
    const cudaError_t ef = cudaFreeAsync(t.T, st);
    return e != cudaSuccess ? e : ef;
  }
  const uint64_t blocks = ((g.P + kBwdPoints - 1) / kBwdPoints) * ((g.S + kBwdTile - 1) / kBwdTile);
  if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float) * ((size_t)g.B * kBwdTile + kBwdPoints * 8);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, sc.device);
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  bwd_kernel<<<(unsigned)blocks, 256, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace nlos
