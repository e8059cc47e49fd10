// Device core of the forward transient: the (scan point, surface point)
// pair sum of the generalised Eq. 1 of Shi et al. (arXiv 2506.03747),
// accumulated per scan point as a histogram over time bins, with the Gaussian
// jitter of Eq. 16/17 fused into the write-out, or as the differentiable
// Gaussian splat. Shared by the standalone forward kernel (forward.cu) and
// the persistent serving kernel (serve.cu), so both run identical arithmetic.
//
// Layout and schedule (GB300, sm_103a):
//  * One tile = 32 scan points; lane l of every warp owns scan point l of the
//    tile, so the shared histogram [bin][32] gives every lane its own bank and
//    the shared atomics of a warp never conflict.
//  * Surface points are packed in pairs (64 B, PointPair) and staged into
//    shared memory by 1-D TMA bulk copies, double-buffered on mbarriers. All
//    warps of the CTA read the same staged block (broadcast loads) and split
//    its pairs; each lane evaluates the two points of a pair for its scan
//    point with packed FP32x2 arithmetic (__ffma2_rn & co.).
//  * A work unit is (scan tile, bin window, point block). A CTA runs a
//    contiguous range of units and flushes its partial histogram into the
//    zeroed output with vectorised global reductions whenever its (tile,
//    window) changes; the jitter convolution is linear, so it is applied to
//    each partial histogram during the flush.
#pragma once

#include "common.cuh"
#include "device_util.cuh"

#include <cmath>

namespace nlos {

constexpr float kMagic = 12582912.0f;       // 1.5 * 2^23: floor via round-down add
constexpr int kMagicBits = 0x4B400000;      // bit pattern of kMagic
constexpr int kMaxTaps = 129;               // fused jitter: R <= 64
constexpr int kPairsPerBlock = 256;         // serving kernel: 16 KB per staged block
#ifndef NLOS_FWD_PPB
#define NLOS_FWD_PPB 512                    // standalone forward: pairs per staged block
#endif
#ifndef NLOS_FWD_ONE_CTA
#define NLOS_FWD_ONE_CTA 1                  // standalone forward: 1 CTA x 1024 threads per SM
#endif
#ifndef NLOS_FWD_SQRT_RCP
#define NLOS_FWD_SQRT_RCP 1                 // r from sqrt.approx, weights from one rcp.approx
#endif
#ifndef NLOS_FWD_CULL
#define NLOS_FWD_CULL 1                     // skip (tile, block) units the bounds rule out
#endif
#ifndef NLOS_FWD_EARLY
#define NLOS_FWD_EARLY 0                    // warp-uniform early out before the square roots
#endif
#ifndef NLOS_FWD_VOTE
#define NLOS_FWD_VOTE 0                     // 2: warp-uniform skip before the reductions
#endif
#ifndef NLOS_FWD_CHUNKS_PER_CTA
#define NLOS_FWD_CHUNKS_PER_CTA 32          // standalone forward: claimed chunks per CTA (mean)
#endif
#ifndef NLOS_FWD_LIST_CHUNKS_PER_CTA
#define NLOS_FWD_LIST_CHUNKS_PER_CTA 6      // live-unit list: chunks per CTA (mean)
#endif
#ifndef NLOS_FWD_LIST_MIN
#define NLOS_FWD_LIST_MIN 2                 // live-unit list: entries per chunk, at least
#endif
#ifndef NLOS_FWD_LIST_STATIC
#define NLOS_FWD_LIST_STATIC 75             // live-unit list: percent in static ranges per CTA
#endif
#ifndef NLOS_FWD_LIST_HALVES
#define NLOS_FWD_LIST_HALVES 1              // live-unit list: halves of a unit culled apart
#endif
#ifndef NLOS_FWD_LIST_MAX
#define NLOS_FWD_LIST_MAX 32                // ... and at most
#endif
#ifndef NLOS_FWD_CONTIG
#define NLOS_FWD_CONTIG 1                   // each warp takes a contiguous run of a block's pairs
#endif
#ifndef NLOS_FWD_STAGES
#define NLOS_FWD_STAGES 3                   // staged blocks in flight (warp-specialised)
#endif
#ifndef NLOS_FWD_UNROLL
#define NLOS_FWD_UNROLL 4                   // standalone forward: unroll of the pair loop
#endif

constexpr int kFwdUnroll = NLOS_FWD_UNROLL;  // (#pragma unroll takes no macro)

enum { MODE_NEAREST = 0, MODE_NEAREST_COUNT = 1, MODE_SPLAT = 2, MODE_SPLAT_MOM = 3,
       MODE_NEAREST_OCC = 4 /* NEAREST with the occluder visibility test */ };

// Moment form of the splat (standalone forward, sigma >= 2.5 bins): per bin m
// and scan point, M_n[m] = sum of w c^n over the pairs with floor(u) = m,
// c = 1/2 - (u - m), n < kMoments; at flush time
//   tau[b] = sum_n sum_j D_n[j] M_n[b - j],  D_n[j] = K^(n)(j) / n!,
// the Taylor expansion of the Gaussian K(j + c) about the bin offset j. With
// 6 moments the truncation error is below 2e-6 of the kernel's peak for sigma
// >= 2.5 (3e-7 at sigma = 3.2). Each moment histogram has kMomRows rows
// (window bins plus J on each side).
constexpr int kMoments = 6;
constexpr int kMomRows = 256;
constexpr int kMomMaxJ = 60;
constexpr uint32_t kMomStride = kMomRows * 32 * 4;  // bytes between moment histograms
struct MomTab {
  int J;                                  // taps j = -J..J
  float d[kMoments][2 * kMomMaxJ + 1];    // D_n[j + J]
};

// Fills mt for the unit-area Gaussian of standard deviation s bins (host).
void moment_table(double s, MomTab& mt);

// The moment form is used for splat kernels of at least 2.5 bins standard
// deviation (truncation error <= 1.3e-6 of the peak) whose taps fit MomTab.
inline bool use_moments(double sigma) {
  return sigma >= 2.5 && (int)std::ceil(6.0 * sigma) + 1 <= kMomMaxJ;
}

// Per-thread counters of one forward run, added to the scene scratch at exit.
struct FwdCount {
  unsigned long long boundary = 0;  // pairs within eps of a bin edge (count mode)
  unsigned long long full = 0;      // warp iterations past the early out (x 64 pairs)
  unsigned long long tested = 0;    // warp iterations of staged units (x 64 pairs)
};

struct FwdArgs {
  const PointPair* pairs;
  const ScanPoint* scan;
  float* tau;
  unsigned int* err;
  unsigned long long* boundary;
  unsigned long long* pairs_full;  // pairs past the early out (scene scratch)
  unsigned long long* pairs_tested;  // pairs of staged units (scene scratch)
  const BlockBound* bounds;   // [ceil(n_pairs / kSubPairs)] or null (no unit culling)
  const TileBound* tiles;     // [ceil(S / kTile)]
  unsigned long long* next_chunk;  // standalone launch: chunk counter (zeroed per pass)
  unsigned long long units;   // standalone launch: total units
  unsigned long long chunk;   // standalone launch: units per claimed chunk
  // standalone launch with a unit list (unit_list_kernel): the live units, as
  // unit | rows << 32 (rows: unit_rows), *n_live of them; chunks of the list
  // are claimed instead of chunks of units (null: no list)
  const unsigned long long* unit_list;
  const unsigned long long* n_live;
  uint32_t list_chunks_per_cta;  // list chunks per CTA (mean), of the claimed part
  uint32_t list_min_chunk, list_max_chunk;  // list entries per chunk, clamped
  uint32_t list_static_pct;  // the list's first part (percent) in one contiguous range per CTA
  uint32_t list_halves;      // list entries carry the units' dead halves (ppb = 2 kSubPairs)
  uint32_t n_pairs, S, B, bw, n_win, n_blk, ppb;
  uint32_t stages;   // staged point blocks (standalone warp-specialised kernel)
  float kbin;        // bins per metre of the scanned leg
  int R;             // jitter radius (NEAREST); 0 = none
  float eps;         // boundary-count tolerance (MODE_NEAREST_COUNT)
  float inv2s2;      // splat: 1 / (2 sigma^2)
  float norm;        // splat: 1 / (sigma sqrt(2 pi))
  float reach;       // splat: 6 sigma
  float qstep;       // splat: exp(-1 / sigma^2)
  float taps[kMaxTaps];
  int replicate;     // jitter with the edge bins continued outside the window
  float tail[kMaxTaps / 2 + 1];  // replicate corrections (jitter_tails)
};

struct bool2_t {
  bool x, y;
};

// Path-bin coordinate u and weight w of the two points of a pair for one scan
// spot (sx, sy, 0) with bin offset off (FP32x2: component i = point i).
//   r^2 = (px - sx)^2 + (py - sy)^2 + pz^2,   u = r * kbin + off (+ uoff)
//   cn  = na * (px - sx) + nb * (py - sy) + nc   (object cosine numerator
//         n.(spot - x), prescaled; from the offsets, so nothing cancels)
// Weight by scan and cosine mode (per-point factors folded in at packing):
//   confocal    NONE: kq / r^4        OBJECT: (cn / r^3)^2   WALL: (cn / r^4)^2
//   non-confocal NONE: kq / r^2       OBJECT: cn / r^3       WALL: cn / r^4
// Split in two: pair_geom2 (r^2 and cn: differences and FMAs only) and
// pair_finish2 (square root, u and the weight), so that the caller can skip
// the second part when no lane of the warp can bin either point.
__device__ __forceinline__ void pair_geom2(const PointPair& q, float2 nsx, float2 nsy, float2& r2,
                                           float2& cn) {
  const float2 dx = __fadd2_rn(q.px, nsx);
  const float2 dy = __fadd2_rn(q.py, nsy);
  r2 = __ffma2_rn(dx, dx, q.pz2);
  r2 = __ffma2_rn(dy, dy, r2);
  cn = __ffma2_rn(q.na, dx, q.nc);
  cn = __ffma2_rn(q.nb, dy, cn);
}

// u is formed relative to bin 0 of the transient; callers move it to the
// window by an exact subtraction of the window's first bin (an integer below
// 2^24: in the float for the splat forms, in the integer bin for the binned
// ones), so the bins and splat taps of a pair do not depend on how the bins
// are windowed.
template <int SCAN, int COS>
__device__ __forceinline__ void pair_finish2(const PointPair& q, float2 r2, float2 cn, float2 off,
                                             float2 kbin, float2& u, float2& w) {
  const float2 o = (SCAN == NLOS_CONFOCAL) ? off : __fadd2_rn(off, q.uoff);
#if NLOS_FWD_SQRT_RCP
  // r from the hardware square root; the weight's inverse powers of r from a
  // single reciprocal of r^2k, so no approximation error is raised to a power
  const float2 r = make_float2(sqrt_approx(r2.x), sqrt_approx(r2.y));
  u = __ffma2_rn(r, kbin, o);
  if (SCAN == NLOS_CONFOCAL) {
    if (COS == NLOS_COS_NONE) {
      const float2 d = __fmul2_rn(r2, r2);
      w = __fmul2_rn(q.kq, make_float2(rcp_approx(d.x), rcp_approx(d.y)));
    } else if (COS == NLOS_COS_OBJECT) {
      const float2 d = __fmul2_rn(__fmul2_rn(r2, r2), r2);
      w = __fmul2_rn(__fmul2_rn(cn, cn), make_float2(rcp_approx(d.x), rcp_approx(d.y)));
    } else {
      const float2 d2 = __fmul2_rn(r2, r2);
      const float2 d = __fmul2_rn(d2, d2);
      w = __fmul2_rn(__fmul2_rn(cn, cn), make_float2(rcp_approx(d.x), rcp_approx(d.y)));
    }
  } else {
    if (COS == NLOS_COS_NONE) {
      w = __fmul2_rn(q.kq, make_float2(rcp_approx(r2.x), rcp_approx(r2.y)));
    } else if (COS == NLOS_COS_OBJECT) {
      const float2 d = __fmul2_rn(r2, r);
      w = __fmul2_rn(cn, make_float2(rcp_approx(d.x), rcp_approx(d.y)));
    } else {
      const float2 d = __fmul2_rn(r2, r2);
      w = __fmul2_rn(cn, make_float2(rcp_approx(d.x), rcp_approx(d.y)));
    }
  }
#else
  float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
  // one Newton step on 1/r (e = 1 - r2 ri^2, ri += ri e / 2): the hardware
  // estimate's few-ulp error would otherwise grow to ~1e-6 in the r^-6 weight
  float2 r = __fmul2_rn(r2, ri);
  const float2 e = __ffma2_rn(make_float2(-r.x, -r.y), ri, make_float2(1.0f, 1.0f));
  ri = __ffma2_rn(__fmul2_rn(ri, make_float2(0.5f, 0.5f)), e, ri);
  r = __fmul2_rn(r2, ri);
  u = __ffma2_rn(r, kbin, o);
  float2 ri2 = __fmul2_rn(ri, ri);
  if (SCAN == NLOS_CONFOCAL) {
    if (COS == NLOS_COS_NONE) {
      w = __fmul2_rn(__fmul2_rn(q.kq, ri2), ri2);
    } else if (COS == NLOS_COS_OBJECT) {
      float2 t = __fmul2_rn(cn, __fmul2_rn(ri2, ri));
      w = __fmul2_rn(t, t);
    } else {
      float2 t = __fmul2_rn(cn, __fmul2_rn(ri2, ri2));
      w = __fmul2_rn(t, t);
    }
  } else {
    if (COS == NLOS_COS_NONE) {
      w = __fmul2_rn(q.kq, ri2);
    } else if (COS == NLOS_COS_OBJECT) {
      w = __fmul2_rn(cn, __fmul2_rn(ri2, ri));
    } else {
      w = __fmul2_rn(cn, __fmul2_rn(ri2, ri2));
    }
  }
#endif
}

template <int SCAN, int COS>
__device__ __forceinline__ void pair_eval2(const PointPair& q, float2 nsx, float2 nsy, float2 off,
                                           float2 kbin, float2& u, float2& w, float2& cn) {
  float2 r2;
  pair_geom2(q, nsx, nsy, r2, cn);
  pair_finish2<SCAN, COS>(q, r2, cn, off, kbin, u, w);
}

// Early-out test on r^2, before any square root: can the point land in
// [-margin, lim + margin) bins of the window for this lane? Conservative
// (margin >= 1 bin against a rounding error of ~1e-3 bin); the exact bin
// test follows for the points that pass.
//   confocal:     r in [r_lo, r_hi) with per-lane bounds (r2lo, r2hi = squares)
//   non-confocal: r_lo/hi = base_lo/hi - uoff / kbin (per point and lane)
template <int SCAN>
__device__ __forceinline__ bool2_t may_bin2(const PointPair& q, float2 r2, float2 r2lo, float2 r2hi,
                                            float2 ikbin_neg) {
  if (SCAN == NLOS_CONFOCAL) {
    return bool2_t{r2.x >= r2lo.x && r2.x < r2hi.x, r2.y >= r2lo.y && r2.y < r2hi.y};
  } else {
    // here r2lo / r2hi hold base_lo / base_hi (in metres, per lane)
    const float2 rlo = __ffma2_rn(q.uoff, ikbin_neg, r2lo);
    const float2 rhi = __ffma2_rn(q.uoff, ikbin_neg, r2hi);
    const float2 lo2 = __fmul2_rn(rlo, rlo);
    const float2 hi2 = __fmul2_rn(rhi, rhi);
    return bool2_t{rhi.x > 0.f && r2.x < hi2.x && (rlo.x <= 0.f || r2.x >= lo2.x),
                   rhi.y > 0.f && r2.y < hi2.y && (rlo.y <= 0.f || r2.y >= lo2.y)};
  }
}

__device__ __forceinline__ void load_pair(const PointPair* p, PointPair& q) {
  const float4* v = reinterpret_cast<const float4*>(p);
  float4 a = v[0], b = v[1], c = v[2], d = v[3];
  q.px = make_float2(a.x, a.y);
  q.py = make_float2(a.z, a.w);
  q.pz2 = make_float2(b.x, b.y);
  q.kq = make_float2(b.z, b.w);
  q.na = make_float2(c.x, c.y);
  q.nb = make_float2(c.z, c.w);
  q.nc = make_float2(d.x, d.y);
  q.uoff = make_float2(d.z, d.w);
}

template <int COS>
__device__ __forceinline__ bool facing(float cn) {
  return COS == NLOS_COS_NONE ? true : (cn > 0.0f);
}

// One point's Gaussian splat into this lane's histogram column (bins of the
// window with |b + 1/2 - u| < 6 sigma), taps by the recurrence
// K_{b+1} = K_b * rho_b, rho_{b+1} = rho_b * exp(-1/sigma^2), restarted from a
// direct evaluation every 8 taps: the recurrence's rounding error grows with
// the square of the number of steps (about 1e-4 after 90 taps in FP32).
__device__ __forceinline__ void splat_one(uint32_t col_addr, float u, float w, int lim,
                                          const FwdArgs& a) {
  float lo_f = floorf(u - 0.5f - a.reach) + 1.0f;
  float hi_f = ceilf(u - 0.5f + a.reach) - 1.0f;
  int lo = max(0, (int)lo_f);
  int hi = min(lim - 1, (int)hi_f);
  if (lo > hi) return;
  const float wn = w * a.norm;
  uint32_t addr = col_addr + (uint32_t)lo * (kTile * 4);
  float K = 0.f, rho = 0.f;
  for (int b = lo; b <= hi; ++b) {
    if (((b - lo) & 7) == 0) {
      const float x = (float)b + 0.5f - u;
      K = wn * expf(-x * x * a.inv2s2);
      rho = expf(-(2.0f * x + 1.0f) * a.inv2s2);
    }
    red_add_shared(addr, K);
    K *= rho;
    rho *= a.qstep;
    addr += kTile * 4;
  }
}

struct FwdSmem {
  float* hist;                 // [bw][32]
  PointPair* stage;            // [stages][ppb]
  uint64_t* bars;              // full[stages] then empty[stages] (initialised by the caller)
  unsigned long long* units;   // [stages]: the unit staged in each slot
  uint32_t* rows = nullptr;    // [kRowWords] or null: row tracking (see fwd_run_ws)
  unsigned long long* lane_units = nullptr;  // [32]: the producer lanes' units (list mode)
};
// rows: 32 words for the producer's lanes, then one per slot (up to 8 stages)
constexpr int kMaxRangedStages = 8;
constexpr int kRowWords = 32 + kMaxRangedStages;

constexpr unsigned long long kNoUnit = ~0ull;  // end of a run (in FwdSmem::units)

// Scan-point state of the (tile, window) a CTA is working on; lane l of every
// warp holds scan point l of the tile.
struct TileState {
  long long tw = -1;
  uint32_t w0 = 0;
  int lim = 0;  // bins of the current window that lie inside [0, B)
  float2 sx2, sy2, nsx2, nsy2;
  float2 off2;          // bin offset of the scan point, relative to bin 0
  float2 nw02;          // -(first bin of the window)
  uint32_t binbase = kMagicBits;  // bit pattern of kMagic + first bin of the window
  float2 r2lo2, r2hi2;  // early-out bounds (see may_bin2)
};

// Bins beyond the window edges that still matter: 1 for the histogram modes
// (edge pairs of the boundary count), the splat reach + 1, J + 1 for moments.
template <int MODE>
__device__ __forceinline__ float window_margin(const FwdArgs& a, int mom_J) {
  return MODE == MODE_SPLAT ? a.reach + 1.0f
         : MODE == MODE_SPLAT_MOM ? (float)(mom_J + 1)
                                  : 1.0f;
}

__device__ __forceinline__ void load_tile(const FwdArgs& a, long long tw, int lane,
                                          TileState& ts, bool confocal, float margin) {
  const uint32_t tile = (uint32_t)(tw / a.n_win);
  ts.tw = tw;
  ts.w0 = (uint32_t)(tw % a.n_win) * a.bw;
  ts.lim = (int)min(a.bw, a.B - ts.w0);
  const uint32_t s = tile * kTile + lane;
  if (s < a.S) {
    const ScanPoint sp = a.scan[s];
    ts.sx2 = make_float2(sp.sx, sp.sx);
    ts.sy2 = make_float2(sp.sy, sp.sy);
    ts.nsx2 = make_float2(-sp.sx, -sp.sx);
    ts.nsy2 = make_float2(-sp.sy, -sp.sy);
    ts.off2 = make_float2(sp.off, sp.off);
    ts.nw02 = make_float2(-(float)ts.w0, -(float)ts.w0);
    ts.binbase = (uint32_t)kMagicBits + ts.w0;
    const float o = sp.off - (float)ts.w0;
    // r range of u in [-margin, lim + margin): r = (u - o) / kbin
    const float ik = 1.0f / a.kbin;
    const float rlo = (-margin - o) * ik, rhi = ((float)ts.lim + margin - o) * ik;
    float lo, hi;
    if (confocal) {
      lo = rlo > 0.f ? rlo * rlo : 0.f;
      hi = rhi > 0.f ? rhi * rhi : -1.f;
    } else {
      lo = rlo;  // the point's uoff / kbin is subtracted in may_bin2
      hi = rhi;
    }
    ts.r2lo2 = make_float2(lo, lo);
    ts.r2hi2 = make_float2(hi, hi);
  } else {
    ts.sx2 = ts.sy2 = ts.nsx2 = ts.nsy2 = make_float2(0.f, 0.f);
    ts.off2 = make_float2(-1e30f, -1e30f);  // u -> -inf: never binned
    ts.nw02 = make_float2(0.f, 0.f);
    ts.binbase = (uint32_t)kMagicBits + ts.w0;
    ts.r2lo2 = make_float2(1.f, 1.f);      // empty r ranges
    ts.r2hi2 = make_float2(-1.f, -1.f);
  }
}

// Four output bins o0..o0+3 of one column: each histogram row read once
// (4 + 2R loads into registers), the taps unrolled at compile time.
template <int R>
__device__ __forceinline__ void conv_quad(const FwdArgs& a, const float* hist, int r0, int bw, int c,
                                          float v[4]) {
  float h[4 + 2 * R];
#pragma unroll
  for (int k = 0; k < 4 + 2 * R; ++k) {
    const int b = r0 - R + k;
    h[k] = (b >= 0 && b < bw) ? hist[b * kTile + c] : 0.f;
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float acc = 0.f;
#pragma unroll
    for (int j = -R; j <= R; ++j) acc = fmaf(a.taps[j + R], h[e - j + R], acc);
    v[e] = acc;
  }
}

// Any radius (taps loop at run time).
__device__ __forceinline__ void conv_quad_any(const FwdArgs& a, const float* hist, int r0, int bw,
                                              int c, int R, float v[4]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int bc = r0 + e;  // histogram row of the centre tap
    float acc = 0.f;
    for (int j = -R; j <= R; ++j) {
      const int b = bc - j;
      if (b >= 0 && b < bw) acc = fmaf(a.taps[j + R], hist[b * kTile + c], acc);
    }
    v[e] = acc;
  }
}

template <int R>
__device__ __forceinline__ void flush_quads(const FwdArgs& a, const float* hist, int lo, int nq,
                                            int w0, int R_rt, uint32_t s, int c, int warp_rel,
                                            int n_warps) {
  for (int qi = warp_rel; qi < nq; qi += n_warps) {
    const int o0 = lo + 4 * qi;
    float v[4];
    if (R >= 0) conv_quad<(R >= 0 ? R : 0)>(a, hist, o0 - w0, (int)a.bw, c, v);
    else conv_quad_any(a, hist, o0 - w0, (int)a.bw, c, R_rt, v);
    if (a.replicate) {
      // the taps beyond the first / last bin read that bin (linear, so each
      // partial histogram adds its own share); only the windows holding it
      const int last = (int)a.B - 1;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int o = o0 + e;
        if (w0 == 0 && o < R_rt) v[e] = fmaf(a.tail[o], hist[c], v[e]);
        if (last - w0 < (int)a.bw && last - o >= 0 && last - o < R_rt)
          v[e] = fmaf(a.tail[last - o], hist[(last - w0) * kTile + c], v[e]);
      }
    }
    if (s < a.S && (v[0] != 0.f || v[1] != 0.f || v[2] != 0.f || v[3] != 0.f)) {
      float* dst = a.tau + (size_t)s * a.B + o0;
      if ((a.B & 3u) == 0u) {
        red_add_global_v4(dst, make_float4(v[0], v[1], v[2], v[3]));
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (o0 + e < (int)a.B && o0 + e >= 0) red_add_global(dst + e, v[e]);
      }
    }
  }
}

// Flush the partial histogram of (tile, window) tw into tau (jittered for
// NEAREST): out[o] = sum_j taps[j + R] * hist[o - w0 - j], zero outside the
// window; four consecutive bins per thread, one vector reduction each. Runs
// on the warps [w_first, w_first + n_warps) of the CTA. Radii up to 16 use
// a compile-time unrolled convolution.
// Only histogram rows [rlo, rhi) may be nonzero, so only the output bins
// they reach are written.
template <int MODE>
__device__ __forceinline__ void flush_tile(const FwdArgs& a, long long tw, const float* hist,
                                           int warp_rel, int n_warps, int rlo, int rhi) {
  const uint32_t tile = (uint32_t)(tw / a.n_win);
  const uint32_t win = (uint32_t)(tw % a.n_win);
  const int w0 = (int)(win * a.bw);
  const int R = (MODE == MODE_SPLAT) ? 0 : a.R;
  if (rhi <= rlo) return;
  const int lo = max(0, w0 + rlo - R) & ~3;
  const int hi = min((int)a.B, w0 + rhi + R);
  if (hi <= lo) return;
  const int nq = (hi - lo + 3) >> 2;  // quads of output bins
  const int c = threadIdx.x & 31;
  // the transient (output row) of the lane's scan point; none for the padding
  // lanes of a ragged last tile
  const uint32_t si = tile * kTile + c;
  const uint32_t s = si < a.S ? a.scan[si].row : 0xFFFFFFFFu;
#define NLOS_FLUSH_R(RR) \
  case RR:               \
    flush_quads<RR>(a, hist, lo, nq, w0, R, s, c, warp_rel, n_warps); \
    break;
  switch (R) {
    NLOS_FLUSH_R(0) NLOS_FLUSH_R(1) NLOS_FLUSH_R(2) NLOS_FLUSH_R(3) NLOS_FLUSH_R(4)
    NLOS_FLUSH_R(5) NLOS_FLUSH_R(6) NLOS_FLUSH_R(7) NLOS_FLUSH_R(8) NLOS_FLUSH_R(9)
    NLOS_FLUSH_R(10) NLOS_FLUSH_R(11) NLOS_FLUSH_R(12) NLOS_FLUSH_R(13) NLOS_FLUSH_R(14)
    NLOS_FLUSH_R(15) NLOS_FLUSH_R(16)
    default:
      flush_quads<-1>(a, hist, lo, nq, w0, R, s, c, warp_rel, n_warps);
  }
#undef NLOS_FLUSH_R
}

// All pairs of one staged block for this warp (pairs warp_rel, warp_rel +
// n_warps, ...): evaluate both points of a pair for the lane's scan point and
// add their weights to the lane's histogram column (or splat them).
// red.shared.add.f32 [addr + k * kMomStride] of w c^k for the moments k <
// kMoments of one point, predicated on row < rows and a facing cosine.
template <int K>
__device__ __forceinline__ void red_moment(uint32_t addr, float wk, uint32_t ok) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n @p red.shared.add.f32 [%0+%3], %1;\n}\n" ::"r"(addr),
      "f"(wk), "r"(ok), "n"(K * kMomStride)
      : "memory");
}

template <int COS>
__device__ __forceinline__ void red_moments(uint32_t addr, float w, float c, uint32_t row,
                                            uint32_t rows, float cn) {
  static_assert(kMoments == 6, "red_moments is written out for six moments");
  const uint32_t ok = (row < rows && (COS == NLOS_COS_NONE || cn > 0.0f)) ? 1u : 0u;
  float wk = w;
  red_moment<0>(addr, wk, ok);
  wk *= c;
  red_moment<1>(addr, wk, ok);
  wk *= c;
  red_moment<2>(addr, wk, ok);
  wk *= c;
  red_moment<3>(addr, wk, ok);
  wk *= c;
  red_moment<4>(addr, wk, ok);
  wk *= c;
  red_moment<5>(addr, wk, ok);
}

// Visibility of the point S + d from the spot S = (sx, sy, 0) (the detector
// leg of a pair; A = |d|^2 > 0, d.z > 0): false when the segment runs
// strictly inside an occluder for more than o.eta of its length. Spheres: the
// chord in units of A (no division), from |S + t d - c|^2 < r^2; boxes: the
// slab intervals of t, with reciprocal estimates. The threshold is far above
// the FP32 rounding of the chord except for near-tangent segments, which the
// parity tests treat like pairs near a bin edge. Only the occluders of `mask`
// (those the unit's segments can meet, occ_unit_mask) are tested.
__device__ __forceinline__ bool occ_seen(const OccSet& o, uint32_t mask, float sx, float sy,
                                         float dx, float dy, float dz, float A) {
  for (; mask; mask &= mask - 1) {
    const int k = __ffs(mask) - 1;
    const float4 p = o.occ[2 * k], q = o.occ[2 * k + 1];
    if (p.w == 0.f) {
      const float fx = sx - p.x, fy = sy - p.y;
      const float B = fmaf(fx, dx, fmaf(fy, dy, -p.z * dz));
      const float C = fmaf(fx, fx, fmaf(fy, fy, fmaf(p.z, p.z, -q.x * q.x)));
      const float disc = fmaf(B, B, -A * C);
      if (disc > 0.f) {
        const float sq = sqrt_approx(disc);
        const float t0 = fmaxf(-B - sq, 0.f), t1 = fminf(-B + sq, A);
        if (t1 - t0 > o.eta * A) return false;
      }
    } else {
      float t0 = 0.f, t1 = 1.f;
      bool miss = false;
      if (dx != 0.f) {
        const float r = rcp_approx(dx);
        const float ta = (p.x - sx) * r, tb = (q.x - sx) * r;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
      } else {
        miss = !(p.x < sx && sx < q.x);
      }
      if (dy != 0.f) {
        const float r = rcp_approx(dy);
        const float ta = (p.y - sy) * r, tb = (q.y - sy) * r;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
      } else {
        miss = miss || !(p.y < sy && sy < q.y);
      }
      const float rz = rcp_approx(dz);  // the spot is at z = 0, dz > 0
      t0 = fmaxf(t0, p.z * rz);
      t1 = fminf(t1, q.z * rz);
      if (!miss && t1 - t0 > o.eta) return false;
    }
  }
  return true;
}

template <int SCAN, int COS, int MODE, int UNROLL>
__device__ __forceinline__ void compute_block(const FwdArgs& a, const PointPair* blkp, uint32_t n,
                                              int warp_rel, int n_warps, const TileState& ts,
                                              uint32_t col_addr, FwdCount& cnt,
                                              int mom_J = 0, const OccSet* occ = nullptr,
                                              uint32_t occ_mask = 0, uint32_t rot = 0) {
  const float2 kbin2 = make_float2(a.kbin, a.kbin);
  const float2 magic2 = make_float2(kMagic, kMagic);
  const float2 ikbin_neg = make_float2(-1.0f / a.kbin, -1.0f / a.kbin);
#if NLOS_FWD_CONTIG
  // a contiguous run of pairs per warp: neighbouring points, so the warps'
  // shared reductions meet different histogram rows at any one time; the
  // short last run rotates over the warps from block to block (rot)
  const uint32_t per = (n + (uint32_t)n_warps - 1u) / (uint32_t)n_warps;
  const uint32_t run = ((uint32_t)warp_rel + rot) % (uint32_t)n_warps;
  const uint32_t i_begin = min(n, run * per), i_end = min(n, i_begin + per), i_step = 1u;
#else
  const uint32_t i_begin = (uint32_t)warp_rel, i_end = n, i_step = (uint32_t)n_warps;
#endif
  // iterations of this warp (counted once per block, not per iteration)
  const uint32_t n_it = i_end > i_begin ? (i_end - 1u - i_begin) / i_step + 1u : 0u;
  cnt.tested += n_it;
#if !NLOS_FWD_EARLY
  cnt.full += n_it;
#endif
#pragma unroll UNROLL
  for (uint32_t i = i_begin; i < i_end; i += i_step) {
    PointPair q;
    load_pair(blkp + i, q);
    float2 r2, cn;
    pair_geom2(q, ts.nsx2, ts.nsy2, r2, cn);
#if NLOS_FWD_EARLY
    // warp-uniform early out: for most (tile, point) combinations of a
    // scene no lane can bin either point (outside the window or facing away).
    // Not in the boundary-count mode, which counts every pair near a bin
    // edge of the whole transient (facing or not) in the first window's pass.
    if (MODE != MODE_NEAREST_COUNT) {
      const bool2_t m = may_bin2<SCAN>(q, r2, ts.r2lo2, ts.r2hi2, ikbin_neg);
      if (!__any_sync(0xffffffffu, (m.x && facing<COS>(cn.x)) || (m.y && facing<COS>(cn.y))))
        continue;
    }
    ++cnt.full;
#endif
    float2 u, w;
    pair_finish2<SCAN, COS>(q, r2, cn, ts.off2, kbin2, u, w);
    // window-relative u for the splat forms (exact: w0 is an integer < 2^24)
    if (MODE == MODE_SPLAT || MODE == MODE_SPLAT_MOM) u = __fadd2_rn(u, ts.nw02);
    if (MODE == MODE_SPLAT) {
      if (facing<COS>(cn.x)) splat_one(col_addr, u.x, w.x, ts.lim, a);
      if (facing<COS>(cn.y)) splat_one(col_addr, u.y, w.y, ts.lim, a);
    } else if (MODE == MODE_SPLAT_MOM) {
      const float2 t = __fadd2_rd(u, magic2);                        // kMagic + floor(u)
      const float2 fl = __fadd2_rn(t, make_float2(-kMagic, -kMagic));  // floor(u), exact
      const float2 fr = __fadd2_rn(u, make_float2(-fl.x, -fl.y));      // u - floor(u), exact
      const float2 c = __fadd2_rn(make_float2(0.5f, 0.5f), make_float2(-fr.x, -fr.y));
      const uint32_t ra = (uint32_t)(__float_as_int(t.x) - kMagicBits + mom_J);
      const uint32_t rb = (uint32_t)(__float_as_int(t.y) - kMagicBits + mom_J);
      const uint32_t rows = (uint32_t)(a.bw + 2 * mom_J);
#if NLOS_FWD_VOTE == 2
      // one warp-uniform test first: most pairs of a tile fall outside the
      // window or face away together
      const bool oka = ra < rows && facing<COS>(cn.x);
      const bool okb = rb < rows && facing<COS>(cn.y);
      if (__any_sync(0xffffffffu, oka || okb)) {
        red_moments<COS>(col_addr + ra * (kTile * 4), w.x, c.x, ra, rows, cn.x);
        red_moments<COS>(col_addr + rb * (kTile * 4), w.y, c.y, rb, rows, cn.y);
      }
#else
      red_moments<COS>(col_addr + ra * (kTile * 4), w.x, c.x, ra, rows, cn.x);
      red_moments<COS>(col_addr + rb * (kTile * 4), w.y, c.y, rb, rows, cn.y);
#endif
    } else {
      // kMagic + floor(u), exactly; the window's first bin comes off the
      // integer (floor(u) - w0 = floor(u - w0) for an integer w0)
      const float2 t = __fadd2_rd(u, magic2);
      uint32_t ba = (uint32_t)__float_as_int(t.x) - ts.binbase;
      uint32_t bb = (uint32_t)__float_as_int(t.y) - ts.binbase;
      if (MODE == MODE_NEAREST_OCC) {
        // visibility only for pairs that would be binned; a hidden pair's bin
        // is moved out of range, so its reduction is predicated off
        const float sx = ts.sx2.x, sy = ts.sy2.x;
        if (ba < (uint32_t)ts.lim && facing<COS>(cn.x) &&
            !occ_seen(*occ, occ_mask, sx, sy, q.px.x - sx, q.py.x - sy, sqrt_approx(q.pz2.x),
                      r2.x))
          ba = 0xFFFFFFFFu;
        if (bb < (uint32_t)ts.lim && facing<COS>(cn.y) &&
            !occ_seen(*occ, occ_mask, sx, sy, q.px.y - sx, q.py.y - sy, sqrt_approx(q.pz2.y),
                      r2.y))
          bb = 0xFFFFFFFFu;
      }
      const uint32_t aa = col_addr + ba * (kTile * 4);
      const uint32_t ab = col_addr + bb * (kTile * 4);
      // the in-window and facing test and the reduction in one predicated
      // block (shared f32 reductions are a compare-and-swap loop here)
#if NLOS_FWD_VOTE == 2
      // preceded by one warp-uniform test: most pairs of a tile fall outside
      // the window or face away together
      const bool oka = ba < (uint32_t)ts.lim && facing<COS>(cn.x);
      const bool okb = bb < (uint32_t)ts.lim && facing<COS>(cn.y);
#endif
#if NLOS_FWD_VOTE == 2
      if (__any_sync(0xffffffffu, oka || okb)) {
        if (COS == NLOS_COS_NONE) {
          red_add_shared_if_bin(aa, w.x, ba, (uint32_t)ts.lim);
          red_add_shared_if_bin(ab, w.y, bb, (uint32_t)ts.lim);
        } else {
          red_add_shared_if_bin_cos(aa, w.x, ba, (uint32_t)ts.lim, cn.x);
          red_add_shared_if_bin_cos(ab, w.y, bb, (uint32_t)ts.lim, cn.y);
        }
      }
#else
      if (COS == NLOS_COS_NONE) {
        red_add_shared_if_bin(aa, w.x, ba, (uint32_t)ts.lim);
        red_add_shared_if_bin(ab, w.y, bb, (uint32_t)ts.lim);
      } else {
        red_add_shared_if_bin_cos(aa, w.x, ba, (uint32_t)ts.lim, cn.x);
        red_add_shared_if_bin_cos(ab, w.y, bb, (uint32_t)ts.lim, cn.y);
      }
#endif
      if (MODE == MODE_NEAREST_COUNT && ts.w0 == 0) {
        // pairs with u within eps of a bin edge m in [0, B] (u is global here)
        const float2 fl = __fadd2_rn(t, make_float2(-kMagic, -kMagic));
        const float fa = u.x - fl.x, fb = u.y - fl.y;
        const bool na = (fa < a.eps && fl.x >= 0.f && fl.x <= (float)a.B) ||
                        (1.0f - fa < a.eps && fl.x + 1.0f >= 0.f && fl.x + 1.0f <= (float)a.B);
        const bool nb = (fb < a.eps && fl.y >= 0.f && fl.y <= (float)a.B) ||
                        (1.0f - fb < a.eps && fl.y + 1.0f >= 0.f && fl.y + 1.0f <= (float)a.B);
        // the odd slot of the last pair may be padding (pz2 huge): its u is
        // never near a valid edge
        cnt.boundary += (unsigned)na + (unsigned)nb;
      }
    }
  }
}

// Moment flush: out[o] = sum_n sum_j D_n[j] M_n[o - w0 - j + J] for the bins o
// of the window inside [0, B); four bins per thread, one vector reduction.
__device__ __forceinline__ void flush_tile_mom(const FwdArgs& a, const MomTab& mt, long long tw,
                                               const float* hist, int warp_rel, int n_warps) {
  const uint32_t tile = (uint32_t)(tw / a.n_win);
  const uint32_t win = (uint32_t)(tw % a.n_win);
  const int w0 = (int)(win * a.bw);
  const int lim = (int)min(a.bw, a.B - (uint32_t)w0);
  const int J = mt.J;
  const int nq = (lim + 3) >> 2;
  const int c = threadIdx.x & 31;
  // the transient (output row) of the lane's scan point; none for the padding
  // lanes of a ragged last tile
  const uint32_t si = tile * kTile + c;
  const uint32_t s = si < a.S ? a.scan[si].row : 0xFFFFFFFFu;
  for (int qi = warp_rel; qi < nq; qi += n_warps) {
    const int r0 = 4 * qi;  // window-relative output bin
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < kMoments; ++k) {
      const float* mk = hist + (size_t)k * kMomRows * kTile;
      const float* dk = mt.d[k];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float acc = v[e];
        // row of tap j: (r0 + e) - j + J, j = -J..J
        for (int j = -J; j <= J; ++j) acc = fmaf(dk[j + J], mk[(r0 + e - j + J) * kTile + c], acc);
        v[e] = acc;
      }
    }
    const int o0 = w0 + r0;
    if (s < a.S && (v[0] != 0.f || v[1] != 0.f || v[2] != 0.f || v[3] != 0.f)) {
      float* dst = a.tau + (size_t)s * a.B + o0;
      if ((a.B & 3u) == 0u && (o0 & 3) == 0) {
        red_add_global_v4(dst, make_float4(v[0], v[1], v[2], v[3]));
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (r0 + e < lim) red_add_global(dst + e, v[e]);
      }
    }
  }
}

__device__ __forceinline__ void issue_block(const FwdArgs& a, const FwdSmem& sm,
                                            unsigned long long unit, int slot) {
  const uint32_t blk = (uint32_t)(unit % a.n_blk);
  const uint32_t first = blk * a.ppb;
  const uint32_t n = min(a.ppb, a.n_pairs - first);
  const uint32_t bytes = n * (uint32_t)sizeof(PointPair);
  mbar_arrive_expect_tx(&sm.bars[slot], bytes);
  bulk_g2s(sm.stage + (size_t)slot * a.ppb, a.pairs + first, bytes, &sm.bars[slot]);
}

// max of a * b over a in [a0, a1], b in [b0, b1]
__device__ __forceinline__ float imax(float a0, float a1, float b0, float b1) {
  return fmaxf(fmaxf(a0 * b0, a0 * b1), fmaxf(a1 * b0, a1 * b1));
}

// Can unit (tile, window, point block) bin anything? From the block's
// bounds and the tile's: the range of u over every (spot, point) of the
// unit (distance bounds between the spot box at z = 0 and the point box)
// against the window with `margin` bins on each side, the object cosine
// (upper bound of n.(spot - x) over the boxes) and whether any point carries
// weight. Conservative: a unit it keeps may still bin nothing.
// Bounds of point block blk: the union of its sub-blocks' bounds.
__device__ __forceinline__ BlockBound block_bound(const FwdArgs& a, uint32_t blk) {
  const uint32_t sub_per = a.ppb / kSubPairs;
  const uint32_t sb0 = blk * sub_per;
  const uint32_t n_sub = (a.n_pairs + kSubPairs - 1) / kSubPairs;
  BlockBound b = a.bounds[sb0];
  for (uint32_t j = 1; j < sub_per && sb0 + j < n_sub; ++j) {
    const BlockBound c = a.bounds[sb0 + j];
    b.x0 = fminf(b.x0, c.x0); b.x1 = fmaxf(b.x1, c.x1);
    b.y0 = fminf(b.y0, c.y0); b.y1 = fmaxf(b.y1, c.y1);
    b.z0 = fminf(b.z0, c.z0); b.z1 = fmaxf(b.z1, c.z1);
    b.nx0 = fminf(b.nx0, c.nx0); b.nx1 = fmaxf(b.nx1, c.nx1);
    b.ny0 = fminf(b.ny0, c.ny0); b.ny1 = fmaxf(b.ny1, c.ny1);
    b.nz0 = fminf(b.nz0, c.nz0); b.nz1 = fmaxf(b.nz1, c.nz1);
    b.uo0 = fminf(b.uo0, c.uo0); b.uo1 = fmaxf(b.uo1, c.uo1);
    b.live = fmaxf(b.live, c.live);
  }
  return b;
}

// Can a point inside the bounds b reach the window starting at bin w0 (lim
// bins) of a tile with spot bounds t (and face one of its spots)? ulo, uhi:
// the range of u over the two boxes, window-relative.
template <int SCAN, int COS>
__device__ __forceinline__ bool bounds_live(const FwdArgs& a, const TileBound& t,
                                            const BlockBound& b, uint32_t w0, float lim,
                                            float margin, float& ulo_out, float& uhi_out) {
  if (b.live == 0.f) return false;
  const float dx = fmaxf(0.f, fmaxf(b.x0 - t.sx1, t.sx0 - b.x1));
  const float dy = fmaxf(0.f, fmaxf(b.y0 - t.sy1, t.sy0 - b.y1));
  const float rmin = sqrtf(dx * dx + dy * dy + b.z0 * b.z0);
  const float fx = fmaxf(fabsf(b.x1 - t.sx0), fabsf(t.sx1 - b.x0));
  const float fy = fmaxf(fabsf(b.y1 - t.sy0), fabsf(t.sy1 - b.y0));
  const float rmax = sqrtf(fx * fx + fy * fy + b.z1 * b.z1);
  float ulo = fmaf(rmin, a.kbin, t.off0) - (float)w0;
  float uhi = fmaf(rmax, a.kbin, t.off1) - (float)w0;
  if (SCAN != NLOS_CONFOCAL) {
    ulo += b.uo0;
    uhi += b.uo1;
  }
  ulo_out = ulo;
  uhi_out = uhi;
  if (uhi < -margin || ulo >= lim + margin) return false;
  if (COS != NLOS_COS_NONE) {
    const float f = imax(b.nx0, b.nx1, t.sx0 - b.x1, t.sx1 - b.x0) +
                    imax(b.ny0, b.ny1, t.sy0 - b.y1, t.sy1 - b.y0) +
                    imax(b.nz0, b.nz1, -b.z1, -b.z0);
    if (f <= 0.f) return false;
  }
  return true;
}

template <int SCAN, int COS>
__device__ __forceinline__ bool unit_live(const FwdArgs& a, unsigned long long unit, float margin,
                                          float& ulo_out, float& uhi_out) {
  const unsigned long long tw = unit / a.n_blk;
  const uint32_t blk = (uint32_t)(unit - tw * a.n_blk);
  const uint32_t tile = (uint32_t)(tw / a.n_win);
  const uint32_t w0 = (uint32_t)(tw % a.n_win) * a.bw;
  const float lim = (float)min(a.bw, a.B - w0);
  const TileBound t = a.tiles[tile];
  const BlockBound b = block_bound(a, blk);
  return bounds_live<SCAN, COS>(a, t, b, w0, lim, margin, ulo_out, uhi_out);
}

// The same test on each half of a two-sub-block unit: whether the unit is
// live, its u range over its live halves, and the halves that are not
// (dead bit h: no pair of half h can reach the window or face a spot).
template <int SCAN, int COS>
__device__ __forceinline__ bool unit_live_halves(const FwdArgs& a, unsigned long long unit,
                                                 float margin, float& ulo_out, float& uhi_out,
                                                 uint32_t& dead) {
  const unsigned long long tw = unit / a.n_blk;
  const uint32_t blk = (uint32_t)(unit - tw * a.n_blk);
  const uint32_t tile = (uint32_t)(tw / a.n_win);
  const uint32_t w0 = (uint32_t)(tw % a.n_win) * a.bw;
  const float lim = (float)min(a.bw, a.B - w0);
  const TileBound t = a.tiles[tile];
  const uint32_t sb0 = blk * 2u;
  const uint32_t n_sub = (a.n_pairs + kSubPairs - 1) / kSubPairs;
  float l0 = 0.f, h0 = 0.f, l1 = 0.f, h1 = 0.f;
  const bool live0 = bounds_live<SCAN, COS>(a, t, a.bounds[sb0], w0, lim, margin, l0, h0);
  const bool live1 = sb0 + 1 < n_sub &&
                     bounds_live<SCAN, COS>(a, t, a.bounds[sb0 + 1], w0, lim, margin, l1, h1);
  dead = (live0 ? 0u : 1u) | (live1 ? 0u : 2u);
  ulo_out = live0 ? (live1 ? fminf(l0, l1) : l0) : l1;
  uhi_out = live0 ? (live1 ? fmaxf(h0, h1) : h0) : h1;
  return live0 || live1;
}

// Occluders that can meet a segment from a spot of the unit's tile (z = 0)
// to a point of its block, as bits (conservative). A segment ending at depth
// z_p in [z0, z1] is at depth zeta at t = zeta / z_p, over the lateral box
// interpolated at t between the tile's spot box and the block's box; over
// the depths an occluder spans, t stays in [zeta_lo / z1, min(1, zeta_hi /
// z0)], and the box is linear in t, so its extremes sit at those two ends.
// Without bounds every occluder counts.
__device__ __forceinline__ uint32_t occ_unit_mask(const FwdArgs& a, unsigned long long unit,
                                                  const OccSet& o) {
  const uint32_t all = o.n >= 32 ? 0xFFFFFFFFu : (1u << o.n) - 1u;
  if (a.bounds == nullptr) return all;
  const unsigned long long tw = unit / a.n_blk;
  const uint32_t blk = (uint32_t)(unit - tw * a.n_blk);
  const TileBound t = a.tiles[(uint32_t)(tw / a.n_win)];
  const BlockBound b = block_bound(a, blk);
  if (!(b.z0 > 0.f)) return all;
  constexpr float pad = 1e-4f;  // metres, against rounding of the boxes
  uint32_t m = 0;
  for (int k = 0; k < o.n; ++k) {
    const float4 p = o.occ[2 * k], q = o.occ[2 * k + 1];
    const bool sph = p.w == 0.f;
    const float ox0 = (sph ? p.x - q.x : p.x) - pad, ox1 = (sph ? p.x + q.x : q.x) + pad;
    const float oy0 = (sph ? p.y - q.x : p.y) - pad, oy1 = (sph ? p.y + q.x : q.y) + pad;
    const float oz0 = (sph ? p.z - q.x : p.z) - pad, oz1 = (sph ? p.z + q.x : q.z) + pad;
    const float zlo = fmaxf(oz0, 0.f), zhi = fminf(oz1, b.z1);
    if (zlo > zhi) continue;
    const float tlo = zlo / b.z1, thi = fminf(1.f, zhi / b.z0);
    const float xmin = fminf(fmaf(tlo, b.x0 - t.sx0, t.sx0), fmaf(thi, b.x0 - t.sx0, t.sx0));
    const float xmax = fmaxf(fmaf(tlo, b.x1 - t.sx1, t.sx1), fmaf(thi, b.x1 - t.sx1, t.sx1));
    const float ymin = fminf(fmaf(tlo, b.y0 - t.sy0, t.sy0), fmaf(thi, b.y0 - t.sy0, t.sy0));
    const float ymax = fmaxf(fmaf(tlo, b.y1 - t.sy1, t.sy1), fmaf(thi, b.y1 - t.sy1, t.sy1));
    if (xmax < ox0 || xmin > ox1 || ymax < oy0 || ymin > oy1) continue;
    m |= 1u << k;
  }
  return m;
}

// Histogram rows a unit can touch, packed lo | hi << 16, from its u range
// (window-relative) widened by the mode's margin and two bins against
// rounding, clipped to [0, bw).
__device__ __forceinline__ uint32_t unit_rows(float ulo, float uhi, float margin, uint32_t bw) {
  const float m = ceilf(margin) + 2.f;
  const float lo = fmaxf(floorf(fmaxf(ulo, -1e6f)) - m, 0.f);
  const float hi = fminf(ceilf(fminf(uhi, 1e6f)) + m + 1.f, (float)bw);
  return lo < hi ? (uint32_t)lo | ((uint32_t)hi << 16) : 0u;
}

// Units carry the occluder mask of MODE_NEAREST_OCC in their top bits.
constexpr int kUnitBits = 48;
constexpr unsigned long long kUnitMask = (1ull << kUnitBits) - 1ull;
// A staged unit's dead halves (unit_live_halves) in tag bits 46-47, and in
// bits 30-31 of a live-unit list entry (whose units are then below 2^30).
constexpr int kHalfShift = 46;
constexpr unsigned long long kUnitIdMask = (1ull << kHalfShift) - 1ull;
constexpr int kListHalfShift = 30;
constexpr uint32_t kListUnitMask = (1u << kListHalfShift) - 1u;

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Warp-specialised run of work units (tile, window, point block) of one job:
// warp 0 (one lane) stages point blocks with TMA bulk copies into `stages`
// slots, the other warps evaluate them. The producer writes each slot's unit
// number beside it (kNoUnit ends the run); the full barrier orders that write
// before the consumers read it. Units come either from the range [u0, u1)
// (chunk_counter == nullptr) or in chunks of `chunk` units claimed from
// *chunk_counter until units_total is reached (or, with max_claims > 0, after
// that many claims), so that CTAs that meet cheap units (culled, or most
// pairs stopped by the early out) take more of them. Consumers
// flush their (tile, window) histogram whenever the tile changes and at the
// end. `it` carries the barrier phases across calls (the serving kernel runs
// one call per work item). UNROLL: unroll of the consumers' pair loop;
// RANGED: track the histogram rows each tile can touch (from the unit
// bounds) and flush and zero only those (both cost registers). Every wait is
// bounded; returns false if one gave up (the error is in *a.err).
template <int SCAN, int COS, int MODE, int UNROLL, bool RANGED>
__device__ bool fwd_run_ws(const FwdArgs& a, unsigned long long u0, unsigned long long u1,
                           const FwdSmem& sm, int stages, FwdCount& cnt, const MomTab* mt,
                           uint32_t& it, unsigned long long* chunk_counter = nullptr,
                           unsigned long long chunk = 0, unsigned long long units_total = 0,
                           uint32_t max_claims = 0, const OccSet* occ = nullptr) {
  const int mom_J = (MODE == MODE_SPLAT_MOM) ? mt->J : 0;
  const uint32_t hist_words = (MODE == MODE_SPLAT_MOM) ? (uint32_t)kMoments * kMomRows * kTile
                                                       : a.bw * kTile;
  __shared__ int s_abort;
  __shared__ uint32_t s_used;  // slots this call used (units + the end mark)
  __shared__ unsigned long long s_list_base;  // first entry of the list's claimed part
  // rows each lane's unit can touch (producer), and for each slot the rows
  // its tile's units so far can touch (consumers), in the caller's shared
  // memory (static arrays here would be repeated in every instantiation)
  uint32_t* const s_lane_rows = sm.rows;
  uint32_t* const s_slot_rows = sm.rows + 32;
  float* hist = sm.hist;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int ncw = (blockDim.x >> 5) - 1;  // consumer warps
  uint64_t* full = sm.bars;
  uint64_t* empty = sm.bars + stages;
  unsigned long long* unit_of = sm.units;
  if (tid == 0) {
    s_abort = 0;
    s_used = 0;
  }
  __syncthreads();
  const bool cull = NLOS_FWD_CULL && a.bounds != nullptr && MODE != MODE_NEAREST_COUNT;
  // histogram rows tracked per tile (flush and zero only those); the moment
  // histograms have their own layout and are always handled whole
  const bool ranged = RANGED && sm.rows != nullptr && cull && MODE != MODE_SPLAT_MOM &&
                      stages <= kMaxRangedStages;
  if (warp == 0) {
    // The whole warp walks the units 32 at a time: each lane tests one unit
    // against the bounds (unit_live), then lane 0 stages the live ones in
    // order. Chunk claims (lane 0) run one ahead of their use.
    const float margin = window_margin<MODE>(a, mom_J);
    // list mode: chunks of the live-unit list, sized from its length
    const bool listed = a.unit_list != nullptr && chunk_counter != nullptr &&
                        sm.lane_units != nullptr;
    // the list's first list_static_pct percent goes to the CTAs in equal
    // contiguous ranges (the list holds each (tile, window)'s units together,
    // so a CTA meets few tiles there); the rest is claimed chunk by chunk
    // (the claimed part's first entry is kept in shared memory: it is read
    // once per claim, and a register for it spilled in the pair loop)
    if (lane == 0) s_list_base = 0;
    __syncwarp();
    if (listed) {
      units_total = *reinterpret_cast<const volatile unsigned long long*>(a.n_live);
      if (lane == 0) s_list_base = units_total * a.list_static_pct / 100ull;
      __syncwarp();
      chunk = (units_total - s_list_base) /
              ((unsigned long long)gridDim.x * a.list_chunks_per_cta);
      chunk = min(max(chunk, (unsigned long long)a.list_min_chunk),
                  (unsigned long long)a.list_max_chunk);
    }
    unsigned long long cur = u0, lim = u1, next = 0;
    bool have_next = false;  // a chunk claimed ahead of its use
    uint32_t claims = 0;
    auto claim = [&]() {
      unsigned long long c = 0;
      if (lane == 0) c = atomicAdd(chunk_counter, 1ull);
      ++claims;
      return __shfl_sync(0xffffffffu, c, 0);
    };
    if (chunk_counter) {
      const unsigned long long base = s_list_base;
      if (base > 0) {
        cur = base * blockIdx.x / gridDim.x;
        lim = base * (blockIdx.x + 1ull) / gridDim.x;
      } else {
        const unsigned long long c = claim();
        cur = min(c * chunk, units_total);
        lim = min(cur + chunk, units_total);
      }
      if (cur < lim && (max_claims == 0 || claims < max_claims)) {
        next = claim();
        have_next = true;
      } else if (cur >= lim && base > 0) {
        // an empty static range: go straight to the claimed part
        const unsigned long long c = claim();
        cur = min(base + c * chunk, units_total);
        lim = min(cur + chunk, units_total);
        if (cur < lim && (max_claims == 0 || claims < max_claims)) {
          next = claim();
          have_next = true;
        }
      }
    }
    uint32_t k = 0;
    bool failed = false;
    long long run_tw = -1;   // lane 0: tile of the last staged unit
    uint32_t run_rows = 0;   // lane 0: union of the rows of that tile's staged units
    for (;;) {
      if (cur == lim && have_next) {
        cur = min(s_list_base + next * chunk, units_total);
        lim = min(cur + chunk, units_total);
        have_next = false;
        if (cur < lim && (max_claims == 0 || claims < max_claims)) {
          next = claim();
          have_next = true;
        }
      }
      if (cur >= lim) break;
      const uint32_t n = (uint32_t)min(32ull, lim - cur);
      bool live;
      if (listed) {
        // every list entry is live; its rows were found with it
        live = lane < n;
        const unsigned long long e = live ? a.unit_list[cur + lane] : 0ull;
        sm.lane_units[lane] = e & 0xFFFFFFFFull;
        if (ranged) s_lane_rows[lane] = (uint32_t)(e >> 32);
        __syncwarp();
      } else {
        float ulo = 0.f, uhi = 0.f;
        live = lane < n && (!cull || unit_live<SCAN, COS>(a, cur + lane, margin, ulo, uhi));
        if (ranged) {
          s_lane_rows[lane] = live ? unit_rows(ulo, uhi, margin, a.bw) : 0u;
          __syncwarp();
        }
      }
      uint32_t mask = __ballot_sync(0xffffffffu, live);
      if (lane == 0) {
        while (mask) {
          const int j = __ffs(mask) - 1;
          mask &= mask - 1;
          const uint32_t g = it + k;  // slot uses continue across calls
          const int slot = (int)(g % (uint32_t)stages);
          const uint32_t use = g / (uint32_t)stages;
          if (use > 0 && !mbar_wait_bounded(&empty[slot], (use - 1) & 1)) {
            atomicOr(a.err, kErrWaitTimeout);
            s_abort = 1;
            failed = true;
            break;
          }
          const unsigned long long raw_unit = listed ? sm.lane_units[j] : cur + j;
          const unsigned long long unit =
              (listed && a.list_halves) ? (raw_unit & kListUnitMask) : raw_unit;
          unsigned long long tag = unit;
          if (listed && a.list_halves)
            tag |= (unsigned long long)(raw_unit >> kListHalfShift) << kHalfShift;
          if (MODE == MODE_NEAREST_OCC)
            tag |= (unsigned long long)occ_unit_mask(a, unit, *occ) << kUnitBits;
          if (ranged) {
            const long long utw = (long long)(unit / a.n_blk);
            const uint32_t ur = s_lane_rows[j];
            if (utw != run_tw) {
              run_tw = utw;
              run_rows = ur;
            } else {
              run_rows = min(run_rows & 0xFFFFu, ur & 0xFFFFu) |
                         (max(run_rows >> 16, ur >> 16) << 16);
            }
            s_slot_rows[slot] = run_rows;
          }
          unit_of[slot] = tag;
          fence_proxy_async_smem();
          issue_block(a, sm, unit, slot);
          ++k;
        }
      }
      if (__shfl_sync(0xffffffffu, (int)failed, 0)) break;
      cur += n;
    }
    if (lane == 0) {
      if (!failed) {
        // end mark: no copy, a plain arrival completes the slot
        const uint32_t g = it + k;
        const int slot = (int)(g % (uint32_t)stages);
        const uint32_t use = g / (uint32_t)stages;
        if (use > 0 && !mbar_wait_bounded(&empty[slot], (use - 1) & 1)) {
          atomicOr(a.err, kErrWaitTimeout);
          s_abort = 1;
        } else {
          unit_of[slot] = kNoUnit;
          mbar_arrive(&full[slot]);
          ++k;
        }
      }
      // copies still in flight must land before the CTA exits or reuses the
      // stages: wait for the last use of every slot (bounded)
      for (uint32_t j = (k > (uint32_t)stages ? k - (uint32_t)stages : 0); j < k; ++j)
        (void)mbar_wait_bounded(&full[(it + j) % (uint32_t)stages],
                                ((it + j) / (uint32_t)stages) & 1);
      s_used = k;
    }
  } else {
    const int cw = warp - 1;
    const int nthr = ncw * 32;
    const uint32_t col_addr = smem_addr(hist) + (uint32_t)lane * 4u;
    TileState ts;
    uint32_t tile_rows = (uint32_t)a.bw << 16;  // rows of the current tile that may be nonzero
    for (uint32_t k = 0;; ++k) {
      const uint32_t g = it + k;
      const int slot = (int)(g % (uint32_t)stages);
      const uint32_t use = g / (uint32_t)stages;
      if (*(volatile int*)&s_abort != 0) break;
      if (!mbar_wait_bounded(&full[slot], use & 1)) {
        if (lane == 0) {
          atomicOr(a.err, kErrWaitTimeout);
          s_abort = 1;
        }
        break;
      }
      const unsigned long long tag = *(volatile unsigned long long*)&unit_of[slot];
      const unsigned long long unit = tag == kNoUnit ? kNoUnit : (tag & kUnitIdMask);
      if (unit != kNoUnit) {
        const long long tw = (long long)(unit / a.n_blk);
        const uint32_t blk = (uint32_t)(unit - (unsigned long long)tw * a.n_blk);
        if (tw != ts.tw) {
          named_barrier(1, nthr);  // every consumer is done with the previous tile
          if (ts.tw >= 0) {
            if (MODE == MODE_SPLAT_MOM) flush_tile_mom(a, *mt, ts.tw, hist, cw, ncw);
            else flush_tile<MODE>(a, ts.tw, hist, cw, ncw, (int)(tile_rows & 0xFFFFu),
                                  (int)(tile_rows >> 16));
            named_barrier(1, nthr);
          }
          // zero what the previous tile may have written (everything the first
          // time: the buffer may hold another item's data)
          const uint32_t z0 = (ranged && ts.tw >= 0) ? (tile_rows & 0xFFFFu) * kTile : 0u;
          const uint32_t z1 = (ranged && ts.tw >= 0) ? (tile_rows >> 16) * kTile : hist_words;
          for (uint32_t i = z0 + tid - 32; i < z1; i += nthr) hist[i] = 0.f;
          load_tile(a, tw, lane, ts, SCAN == NLOS_CONFOCAL, window_margin<MODE>(a, mom_J));
          named_barrier(1, nthr);
        }
        // the producer's running union for this tile, up to this unit
        if (ranged) tile_rows = s_slot_rows[slot];
        const uint32_t first = blk * a.ppb;
        const uint32_t nb = min(a.ppb, a.n_pairs - first);
        // halves of the block the list ruled out are not evaluated
        const uint32_t dead = (uint32_t)(tag >> kHalfShift) & 3u;
        const uint32_t lo = (dead & 1u) ? min(nb, (uint32_t)kSubPairs) : 0u;
        const uint32_t hi = (dead & 2u) ? min(nb, (uint32_t)kSubPairs) : nb;
        compute_block<SCAN, COS, MODE, UNROLL>(a, sm.stage + (size_t)slot * a.ppb + lo,
                                       hi > lo ? hi - lo : 0u, cw, ncw, ts, col_addr, cnt,
                                       mom_J, occ, (uint32_t)(tag >> kUnitBits), g);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
      if (unit == kNoUnit) break;
    }
    named_barrier(1, nthr);
    if (ts.tw >= 0) {
      if (MODE == MODE_SPLAT_MOM) flush_tile_mom(a, *mt, ts.tw, hist, cw, ncw);
      else flush_tile<MODE>(a, ts.tw, hist, cw, ncw, (int)(tile_rows & 0xFFFFu),
                            (int)(tile_rows >> 16));
    }
  }
  __syncthreads();
  it += s_used;
  return s_abort == 0;
}

}  // namespace nlos
