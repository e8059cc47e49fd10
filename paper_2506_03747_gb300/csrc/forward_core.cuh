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

namespace nlos {

constexpr int kTile = 32;                   // scan points per CTA tile
constexpr float kMagic = 12582912.0f;       // 1.5 * 2^23: floor via round-down add
constexpr int kMagicBits = 0x4B400000;      // bit pattern of kMagic
constexpr int kMaxTaps = 129;               // fused jitter: R <= 64
constexpr int kPairsPerBlock = 256;         // serving kernel: 16 KB per staged block
#ifndef NLOS_FWD_PPB
#define NLOS_FWD_PPB 256                    // standalone forward: pairs per staged block
#endif
#ifndef NLOS_FWD_ONE_CTA
#define NLOS_FWD_ONE_CTA 0                  // standalone forward: 1 CTA x 1024 threads per SM
#endif
#ifndef NLOS_FWD_WS
#define NLOS_FWD_WS 1                       // standalone forward: warp-specialised staging
#endif
#ifndef NLOS_FWD_STAGES
#define NLOS_FWD_STAGES 3                   // staged blocks in flight (warp-specialised)
#endif

enum { MODE_NEAREST = 0, MODE_NEAREST_COUNT = 1, MODE_SPLAT = 2 };

struct FwdArgs {
  const PointPair* pairs;
  const ScanPoint* scan;
  float* tau;
  unsigned int* err;
  unsigned long long* boundary;
  unsigned long long units;   // standalone launch: total units
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
};

// Path-bin coordinate u and weight w of the two points of a pair for one scan
// spot (sx, sy, 0) with bin offset off (FP32x2: component i = point i).
//   r^2 = (px - sx)^2 + (py - sy)^2 + pz^2,   u = r * kbin + off (+ uoff)
//   cn  = na * (px - sx) + nb * (py - sy) + nc   (object cosine numerator
//         n.(spot - x), prescaled; from the offsets, so nothing cancels)
// Weight by scan and cosine mode (per-point factors folded in at packing):
//   confocal    NONE: kq / r^4        OBJECT: (cn / r^3)^2   WALL: (cn / r^4)^2
//   non-confocal NONE: kq / r^2       OBJECT: cn / r^3       WALL: cn / r^4
template <int SCAN, int COS>
__device__ __forceinline__ void pair_eval2(const PointPair& q, float2 nsx, float2 nsy, float2 sx,
                                           float2 sy, float2 off, float2 kbin, float2& u,
                                           float2& w, float2& cn) {
  float2 dx = __fadd2_rn(q.px, nsx);
  float2 dy = __fadd2_rn(q.py, nsy);
  float2 r2 = __ffma2_rn(dx, dx, q.pz2);
  r2 = __ffma2_rn(dy, dy, r2);
  float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
  // one Newton step on 1/r (e = 1 - r2 ri^2, ri += ri e / 2): the hardware
  // estimate's few-ulp error would otherwise grow to ~1e-6 in the r^-6 weight
  float2 r = __fmul2_rn(r2, ri);
  const float2 e = __ffma2_rn(make_float2(-r.x, -r.y), ri, make_float2(1.0f, 1.0f));
  ri = __ffma2_rn(__fmul2_rn(ri, make_float2(0.5f, 0.5f)), e, ri);
  r = __fmul2_rn(r2, ri);
  float2 o = (SCAN == NLOS_CONFOCAL) ? off : __fadd2_rn(off, q.uoff);
  u = __ffma2_rn(r, kbin, o);
  cn = __ffma2_rn(q.na, dx, q.nc);
  cn = __ffma2_rn(q.nb, dy, cn);
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
// K_{b+1} = K_b * rho_b, rho_{b+1} = rho_b * exp(-1/sigma^2).
__device__ __forceinline__ void splat_one(uint32_t col_addr, float u, float w, int lim,
                                          const FwdArgs& a) {
  float lo_f = floorf(u - 0.5f - a.reach) + 1.0f;
  float hi_f = ceilf(u - 0.5f + a.reach) - 1.0f;
  int lo = max(0, (int)lo_f);
  int hi = min(lim - 1, (int)hi_f);
  if (lo > hi) return;
  float x0 = (float)lo + 0.5f - u;
  float K = w * a.norm * expf(-x0 * x0 * a.inv2s2);
  float rho = expf(-(2.0f * x0 + 1.0f) * a.inv2s2);
  uint32_t addr = col_addr + (uint32_t)lo * (kTile * 4);
  for (int b = lo; b <= hi; ++b) {
    red_add_shared(addr, K);
    K *= rho;
    rho *= a.qstep;
    addr += kTile * 4;
  }
}

struct FwdSmem {
  float* hist;        // [bw][32]
  PointPair* stage;   // [stages][ppb]
  uint64_t* bars;     // full[stages] then empty[stages] (initialised by the caller)
};

// Scan-point state of the (tile, window) a CTA is working on; lane l of every
// warp holds scan point l of the tile.
struct TileState {
  long long tw = -1;
  uint32_t w0 = 0;
  int lim = 0;  // bins of the current window that lie inside [0, B)
  float2 sx2, sy2, nsx2, nsy2, off2;
};

__device__ __forceinline__ void load_tile(const FwdArgs& a, long long tw, int lane,
                                          TileState& ts) {
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
    const float o = sp.off - (float)ts.w0;
    ts.off2 = make_float2(o, o);
  } else {
    ts.sx2 = ts.sy2 = ts.nsx2 = ts.nsy2 = make_float2(0.f, 0.f);
    ts.off2 = make_float2(-1e30f, -1e30f);  // u -> -inf: never binned
  }
}

// Flush the partial histogram of (tile, window) tw into tau (jittered for
// NEAREST): out[o] = sum_j taps[j + R] * hist[o - w0 - j], zero outside the
// window; four consecutive bins per thread, one vector reduction each. Runs
// on the warps [w_first, w_first + n_warps) of the CTA.
template <int MODE>
__device__ __forceinline__ void flush_tile(const FwdArgs& a, long long tw, const float* hist,
                                           int warp_rel, int n_warps) {
  const uint32_t tile = (uint32_t)(tw / a.n_win);
  const uint32_t win = (uint32_t)(tw % a.n_win);
  const int w0 = (int)(win * a.bw);
  const int R = (MODE == MODE_SPLAT) ? 0 : a.R;
  const int lo = max(0, w0 - R) & ~3;
  const int hi = min((int)a.B, w0 + (int)a.bw + R);
  const int nq = (hi - lo + 3) >> 2;  // quads of output bins
  const int c = threadIdx.x & 31;
  const uint32_t s = tile * kTile + c;
  for (int qi = warp_rel; qi < nq; qi += n_warps) {
    const int o0 = lo + 4 * qi;
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int bc = o0 + e - w0;  // histogram row of the centre tap
      float acc = 0.f;
      for (int j = -R; j <= R; ++j) {
        const int b = bc - j;
        if (b >= 0 && b < (int)a.bw) acc = fmaf(a.taps[j + R], hist[b * kTile + c], acc);
      }
      v[e] = acc;
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

// All pairs of one staged block for this warp (pairs warp_rel, warp_rel +
// n_warps, ...): evaluate both points of a pair for the lane's scan point and
// add their weights to the lane's histogram column (or splat them).
template <int SCAN, int COS, int MODE>
__device__ __forceinline__ void compute_block(const FwdArgs& a, const PointPair* blkp, uint32_t n,
                                              int warp_rel, int n_warps, const TileState& ts,
                                              uint32_t col_addr, unsigned long long& nboundary) {
  const float2 kbin2 = make_float2(a.kbin, a.kbin);
  const float2 magic2 = make_float2(kMagic, kMagic);
#pragma unroll 2
  for (uint32_t i = warp_rel; i < n; i += n_warps) {
    PointPair q;
    load_pair(blkp + i, q);
    float2 u, w, cn;
    pair_eval2<SCAN, COS>(q, ts.nsx2, ts.nsy2, ts.sx2, ts.sy2, ts.off2, kbin2, u, w, cn);
    if (MODE == MODE_SPLAT) {
      if (facing<COS>(cn.x)) splat_one(col_addr, u.x, w.x, ts.lim, a);
      if (facing<COS>(cn.y)) splat_one(col_addr, u.y, w.y, ts.lim, a);
    } else {
      const float2 t = __fadd2_rd(u, magic2);  // kMagic + floor(u), exactly
      const uint32_t ba = (uint32_t)(__float_as_int(t.x) - kMagicBits);
      const uint32_t bb = (uint32_t)(__float_as_int(t.y) - kMagicBits);
      const uint32_t aa = col_addr + ba * (kTile * 4);
      const uint32_t ab = col_addr + bb * (kTile * 4);
      if (COS == NLOS_COS_NONE) {
        red_add_shared_if_bin(aa, w.x, ba, (uint32_t)ts.lim);
        red_add_shared_if_bin(ab, w.y, bb, (uint32_t)ts.lim);
      } else {
        red_add_shared_if_bin_cos(aa, w.x, ba, (uint32_t)ts.lim, cn.x);
        red_add_shared_if_bin_cos(ab, w.y, bb, (uint32_t)ts.lim, cn.y);
      }
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
        nboundary += (unsigned)na + (unsigned)nb;
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

// Runs the work units [u0, u1) of one job (a contiguous range in (tile,
// window, point block) order) on this CTA and flushes its partial histograms
// into a.tau. Two staged blocks, all warps compute, CTA barriers between
// blocks (used by the serving kernel, whose CTAs switch jobs between calls).
// The staging use counter `it_base` carries the mbarrier phases across
// calls. Returns false if a bounded wait gave up (the error is recorded in
// *a.err); every thread returns the same value.
template <int SCAN, int COS, int MODE>
__device__ bool fwd_run(const FwdArgs& a, unsigned long long u0, unsigned long long u1,
                        const FwdSmem& sm, uint32_t& it_base, unsigned long long& nboundary) {
  float* hist = sm.hist;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  if (u0 >= u1) return true;
  if (tid == 0) {
    issue_block(a, sm, u0, it_base & 1);
    if (u0 + 1 < u1) issue_block(a, sm, u0 + 1, (it_base + 1) & 1);
  }
  const uint32_t col_addr = smem_addr(hist) + (uint32_t)lane * 4u;
  TileState ts;
  for (unsigned long long unit = u0; unit < u1; ++unit) {
    const uint32_t it = it_base + (uint32_t)(unit - u0);
    const int slot = it & 1;
    const uint32_t parity = (it >> 1) & 1;
    const long long tw = (long long)(unit / a.n_blk);
    const uint32_t blk = (uint32_t)(unit - (unsigned long long)tw * a.n_blk);
    if (tw != ts.tw) {
      if (ts.tw >= 0) {
        flush_tile<MODE>(a, ts.tw, hist, warp, nwarps);
        __syncthreads();
      }
      for (uint32_t i = tid; i < a.bw * kTile; i += blockDim.x) hist[i] = 0.f;
      load_tile(a, tw, lane, ts);
      __syncthreads();
    }
    const bool ok = mbar_wait_bounded(&sm.bars[slot], parity);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(a.err, kErrWaitTimeout);
        if (unit + 1 < u1) (void)mbar_wait_bounded(&sm.bars[slot ^ 1], ((it + 1) >> 1) & 1);
      }
      it_base += (uint32_t)(u1 - u0);
      return false;
    }
    const uint32_t first = blk * a.ppb;
    compute_block<SCAN, COS, MODE>(a, sm.stage + (size_t)slot * a.ppb, min(a.ppb, a.n_pairs - first),
                                   warp, nwarps, ts, col_addr, nboundary);
    __syncthreads();
    if (tid == 0 && unit + 2 < u1) {
      fence_proxy_async_smem();
      issue_block(a, sm, unit + 2, slot);
    }
  }
  flush_tile<MODE>(a, ts.tw, hist, warp, nwarps);
  __syncthreads();  // histogram reads done before the next call zeroes it
  it_base += (uint32_t)(u1 - u0);
  return true;
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Warp-specialised variant for the standalone kernel (one job per launch):
// warp 0 stages point blocks with TMA into `stages` buffers, the other warps
// compute; a consumer warp releases a buffer by arriving on its "empty"
// mbarrier, so warps never wait for one another between blocks. CTA-wide
// synchronisation (a named barrier over the consumer warps) happens only when
// the (tile, window) changes. Bars: full[0..stages) (count 1 + bytes),
// empty[stages..2 stages) (count = consumer warps). Every wait is bounded; a
// wait that gives up sets *a.err and an abort flag, after which the warps skip
// their work but keep arriving, so no barrier is left waiting.
template <int SCAN, int COS, int MODE>
__device__ void fwd_run_ws(const FwdArgs& a, unsigned long long u0, unsigned long long u1,
                           const FwdSmem& sm, int stages, unsigned long long& nboundary) {
  __shared__ int s_abort;
  float* hist = sm.hist;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int ncw = (blockDim.x >> 5) - 1;  // consumer warps
  uint64_t* full = sm.bars;
  uint64_t* empty = sm.bars + stages;
  if (tid == 0) s_abort = 0;
  __syncthreads();
  const uint32_t nunits = (uint32_t)(u1 - u0);
  if (warp == 0) {
    if (lane == 0) {
      uint32_t k = 0;
      for (; k < nunits; ++k) {
        const int slot = (int)(k % (uint32_t)stages);
        const uint32_t use = k / (uint32_t)stages;
        if (use > 0 && !mbar_wait_bounded(&empty[slot], (use - 1) & 1)) {
          atomicOr(a.err, kErrWaitTimeout);
          s_abort = 1;
          break;
        }
        fence_proxy_async_smem();
        issue_block(a, sm, u0 + k, slot);
      }
      // copies still in flight must land before the CTA can exit: wait for
      // the last use of every stage that was issued (bounded)
      for (uint32_t j = (k > (uint32_t)stages ? k - (uint32_t)stages : 0); j < k; ++j)
        (void)mbar_wait_bounded(&full[j % (uint32_t)stages], (j / (uint32_t)stages) & 1);
    }
  } else {
    const int cw = warp - 1;
    const int nthr = ncw * 32;
    const uint32_t col_addr = smem_addr(hist) + (uint32_t)lane * 4u;
    TileState ts;
    for (uint32_t k = 0; k < nunits; ++k) {
      const unsigned long long unit = u0 + k;
      const int slot = (int)(k % (uint32_t)stages);
      const uint32_t use = k / (uint32_t)stages;
      const long long tw = (long long)(unit / a.n_blk);
      const uint32_t blk = (uint32_t)(unit - (unsigned long long)tw * a.n_blk);
      if (tw != ts.tw) {
        named_barrier(1, nthr);  // every consumer is done with the previous tile
        if (ts.tw >= 0) {
          flush_tile<MODE>(a, ts.tw, hist, cw, ncw);
          named_barrier(1, nthr);
        }
        for (uint32_t i = tid - 32; i < a.bw * kTile; i += nthr) hist[i] = 0.f;
        load_tile(a, tw, lane, ts);
        named_barrier(1, nthr);
      }
      const bool aborted = *(volatile int*)&s_abort != 0;
      if (!aborted) {
        if (mbar_wait_bounded(&full[slot], use & 1)) {
          const uint32_t first = blk * a.ppb;
          compute_block<SCAN, COS, MODE>(a, sm.stage + (size_t)slot * a.ppb,
                                         min(a.ppb, a.n_pairs - first), cw, ncw, ts, col_addr,
                                         nboundary);
        } else if (lane == 0) {
          atomicOr(a.err, kErrWaitTimeout);
          s_abort = 1;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
    }
    named_barrier(1, nthr);
    flush_tile<MODE>(a, ts.tw, hist, cw, ncw);
  }
  __syncthreads();
}

}  // namespace nlos
