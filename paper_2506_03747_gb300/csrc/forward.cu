// Forward transient kernel: the (scan point, surface point) pair sum of the
// generalised Eq. 1 of Shi et al. (arXiv 2506.03747), accumulated as a
// per-scan-point histogram over time bins, with the Gaussian jitter of
// Eq. 16/17 fused into the write-out, or as the differentiable Gaussian splat.
//
// Layout and schedule (GB300, sm_103a):
//  * One CTA tile = 32 scan points; lane l of every warp owns scan point l of
//    the tile, so the shared histogram [bin][32] gives every lane its own bank
//    and the shared atomics of a warp never conflict.
//  * Surface points are packed in pairs (64 B, see PointPair) and staged into
//    shared memory by 1-D TMA bulk copies, double-buffered on mbarriers. All
//    warps of the CTA read the same staged block (broadcast loads) and split
//    its pairs; each lane evaluates the two points of a pair for its scan
//    point with packed FP32x2 arithmetic (__ffma2_rn & co.).
//  * Work units (scan tile, bin window, point block) are split evenly over a
//    persistent grid (stream-K): a CTA flushes its partial histogram into the
//    zeroed output with vectorised global reductions whenever its (tile,
//    window) changes. The jitter convolution is linear, so it is applied to
//    each partial histogram during the flush.
#include "forward_core.cuh"
#include "pack_core.cuh"

#include <algorithm>

namespace nlos {

// Standalone launch: a persistent grid (one CTA per SM) claims chunks of the
// job's work units from a counter in the scene scratch.
template <int SCAN, int COS, int MODE>
__global__ void __launch_bounds__(1024, 1)
    fwd_kernel(const __grid_constant__ FwdArgs a, const __grid_constant__ MomTab mt,
               const __grid_constant__ OccSet occ) {
  extern __shared__ __align__(128) unsigned char smem[];
  FwdSmem sm;
  const size_t hist_bytes = (MODE == MODE_SPLAT_MOM) ? (size_t)kMoments * kMomRows * kTile * 4
                                                     : (size_t)a.bw * kTile * 4;
  sm.hist = reinterpret_cast<float*>(smem);
  sm.stage = reinterpret_cast<PointPair*>(smem + hist_bytes);
  sm.bars = reinterpret_cast<uint64_t*>(sm.stage + (size_t)a.stages * a.ppb);
  sm.units = reinterpret_cast<unsigned long long*>(sm.bars + 2 * a.stages);
  sm.lane_units = sm.units + a.stages + 1;
  sm.rows = reinterpret_cast<uint32_t*>(sm.lane_units + 32);
  if (threadIdx.x == 0) {
    for (uint32_t i = 0; i < a.stages; ++i) {
      mbar_init(&sm.bars[i], 1);                                 // full
      mbar_init(&sm.bars[a.stages + i], (blockDim.x >> 5) - 1);  // empty (consumer warps)
    }
    fence_mbar_init();
  }
  __syncthreads();
  FwdCount cnt;
  uint32_t it = 0;
  (void)fwd_run_ws<SCAN, COS, MODE, kFwdUnroll, true>(a, 0, 0, sm, (int)a.stages, cnt, &mt, it,
                                                      a.next_chunk, a.chunk, a.units, 0, &occ);
  if (MODE == MODE_NEAREST_COUNT && cnt.boundary) atomicAdd(a.boundary, cnt.boundary);
  // the count is warp-uniform: one lane adds it, 64 pairs per warp iteration
  if ((threadIdx.x & 31) == 0 && cnt.full) atomicAdd(a.pairs_full, cnt.full * 64ull);
  if ((threadIdx.x & 31) == 0 && cnt.tested) atomicAdd(a.pairs_tested, cnt.tested * 64ull);
}

// The live units of a pass, for the forward's chunk claims: one CTA per
// (tile, window) tests the point blocks against the bounds (unit_live, as
// the producer warp would) and appends the live ones, with the histogram rows
// they can touch, to the list (unit | rows << 32). Entries of one (tile,
// window) are contiguous, so a chunk of the list rarely spans two tiles; the
// order of the (tile, window) runs in the list does not matter.
template <int SCAN, int COS, int MODE>
__global__ void __launch_bounds__(256) unit_list_kernel(const __grid_constant__ FwdArgs a,
                                                        int mom_J,
                                                        unsigned long long* __restrict__ list,
                                                        unsigned long long* __restrict__ n_live) {
  __shared__ uint32_t s_warp[8];
  __shared__ unsigned long long s_base;
  const unsigned long long tw = blockIdx.x;
  const float margin = window_margin<MODE>(a, mom_J);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t b0 = 0; b0 < a.n_blk; b0 += blockDim.x) {
    const uint32_t blk = b0 + threadIdx.x;
    const unsigned long long unit = tw * a.n_blk + blk;
    float ulo = 0.f, uhi = 0.f;
    uint32_t dead = 0;
    const bool live =
        blk < a.n_blk && (a.list_halves
                              ? unit_live_halves<SCAN, COS>(a, unit, margin, ulo, uhi, dead)
                              : unit_live<SCAN, COS>(a, unit, margin, ulo, uhi));
    const uint32_t rows = live ? unit_rows(ulo, uhi, margin, a.bw) : 0u;
    const uint32_t m = __ballot_sync(0xffffffffu, live);
    if (lane == 0) s_warp[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        const uint32_t c = s_warp[w];
        s_warp[w] = tot;
        tot += c;
      }
      s_base = tot ? atomicAdd(n_live, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    if (live) {
      const uint32_t pos = s_warp[warp] + __popc(m & ((1u << lane) - 1u));
      list[s_base + pos] =
          unit | ((unsigned long long)dead << kListHalfShift) | ((unsigned long long)rows << 32);
    }
    __syncthreads();
  }
}

// Per-pair table (debug/parity): the same pack and pair_eval2 arithmetic on
// the points 2k, 2k + 1 of the caller's order (the forward packs them in a
// spatial order) for scan point s_begin + i; u relative to bin 0, w as
// accumulated.
struct PairTableArgs {
  const float* raw;
  unsigned int* err;
  uint32_t n_pairs, P;
  int scan_mode, cos_mode;
  PackConst pc;
};

template <int SCAN, int COS>
__global__ void pair_table_kernel(const PairTableArgs t, const ScanPoint* scan, uint64_t s_begin,
                                  uint64_t s_count, float kbin, float* u_out, float* w_out) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n_pairs = t.n_pairs, P = t.P;
  if (idx >= s_count * n_pairs) return;
  const uint64_t i = idx / n_pairs;
  const uint32_t k = (uint32_t)(idx % n_pairs);
  const ScanPoint sp = scan[s_begin + i];
  const PointPair q = pack_pair_value(t.raw, P, k, t.scan_mode, t.cos_mode, t.pc, t.err, nullptr);
  float2 u, w, cn;
  pair_eval2<SCAN, COS>(q, make_float2(-sp.sx, -sp.sx), make_float2(-sp.sy, -sp.sy),
                        make_float2(sp.off, sp.off), make_float2(kbin, kbin), u, w, cn);
  if (!facing<COS>(cn.x)) w.x = 0.f;
  if (!facing<COS>(cn.y)) w.y = 0.f;
  const uint64_t p0 = 2ull * k;
  if (u_out) {
    u_out[i * P + p0] = u.x;
    if (p0 + 1 < P) u_out[i * P + p0 + 1] = u.y;
  }
  if (w_out) {
    w_out[i * P + p0] = w.x;
    if (p0 + 1 < P) w_out[i * P + p0 + 1] = w.y;
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
namespace {

using FwdFn = void (*)(FwdArgs, MomTab, OccSet);
using ListFn = void (*)(FwdArgs, int, unsigned long long*, unsigned long long*);

template <int SCAN, int COS>
ListFn pick_list_mode(int mode) {
  switch (mode) {
    case MODE_NEAREST: return unit_list_kernel<SCAN, COS, MODE_NEAREST>;
    case MODE_NEAREST_OCC: return unit_list_kernel<SCAN, COS, MODE_NEAREST_OCC>;
    case MODE_SPLAT_MOM: return unit_list_kernel<SCAN, COS, MODE_SPLAT_MOM>;
    case MODE_SPLAT: return unit_list_kernel<SCAN, COS, MODE_SPLAT>;
    default: return nullptr;  // the boundary count evaluates every unit
  }
}

ListFn pick_list(int scan, int cos, int mode) {
  if (scan == NLOS_CONFOCAL) {
    if (cos == NLOS_COS_NONE) return pick_list_mode<NLOS_CONFOCAL, NLOS_COS_NONE>(mode);
    if (cos == NLOS_COS_OBJECT) return pick_list_mode<NLOS_CONFOCAL, NLOS_COS_OBJECT>(mode);
    return pick_list_mode<NLOS_CONFOCAL, NLOS_COS_OBJECT_WALL>(mode);
  }
  if (cos == NLOS_COS_NONE) return pick_list_mode<NLOS_NONCONFOCAL, NLOS_COS_NONE>(mode);
  if (cos == NLOS_COS_OBJECT) return pick_list_mode<NLOS_NONCONFOCAL, NLOS_COS_OBJECT>(mode);
  return pick_list_mode<NLOS_NONCONFOCAL, NLOS_COS_OBJECT_WALL>(mode);
}

template <int SCAN, int COS>
FwdFn pick_mode(int mode) {
  switch (mode) {
    case MODE_NEAREST: return fwd_kernel<SCAN, COS, MODE_NEAREST>;
    case MODE_NEAREST_COUNT: return fwd_kernel<SCAN, COS, MODE_NEAREST_COUNT>;
    case MODE_NEAREST_OCC: return fwd_kernel<SCAN, COS, MODE_NEAREST_OCC>;
    case MODE_SPLAT_MOM: return fwd_kernel<SCAN, COS, MODE_SPLAT_MOM>;
    default: return fwd_kernel<SCAN, COS, MODE_SPLAT>;
  }
}

FwdFn pick(int scan, int cos, int mode) {
  if (scan == NLOS_CONFOCAL) {
    if (cos == NLOS_COS_NONE) return pick_mode<NLOS_CONFOCAL, NLOS_COS_NONE>(mode);
    if (cos == NLOS_COS_OBJECT) return pick_mode<NLOS_CONFOCAL, NLOS_COS_OBJECT>(mode);
    return pick_mode<NLOS_CONFOCAL, NLOS_COS_OBJECT_WALL>(mode);
  }
  if (cos == NLOS_COS_NONE) return pick_mode<NLOS_NONCONFOCAL, NLOS_COS_NONE>(mode);
  if (cos == NLOS_COS_OBJECT) return pick_mode<NLOS_NONCONFOCAL, NLOS_COS_OBJECT>(mode);
  return pick_mode<NLOS_NONCONFOCAL, NLOS_COS_OBJECT_WALL>(mode);
}

}  // namespace

// D_n[j] = K^(n)(j) / n! for the Gaussian K(x) = exp(-x^2/(2 s^2)) / (s sqrt(2 pi)):
// K^(n)(x) = (-1)^n He_n(x/s) K(x) / s^n with the probabilists' Hermite
// polynomials He_0 = 1, He_1 = t, He_{n+1} = t He_n - n He_{n-1} (FP64).
void moment_table(double s, MomTab& mt) {
  mt.J = (int)std::ceil(6.0 * s) + 1;
  for (int j = -mt.J; j <= mt.J; ++j) {
    const double t = (double)j / s;
    const double k = std::exp(-0.5 * t * t) / (s * std::sqrt(2.0 * 3.14159265358979323846));
    double he[kMoments];
    he[0] = 1.0;
    if (kMoments > 1) he[1] = t;
    for (int n = 1; n + 1 < kMoments; ++n) he[n + 1] = t * he[n] - n * he[n - 1];
    double fact = 1.0, spow = 1.0;
    for (int n = 0; n < kMoments; ++n) {
      if (n >= 1) fact *= n;
      mt.d[n][j + mt.J] = (float)(((n & 1) ? -1.0 : 1.0) * he[n] * k / (spow * fact));
      spow *= s;
    }
  }
}

int jitter_radius(double sigma) {
  if (!(sigma > 0.0)) return 0;
  return (int)std::ceil(2.0 * sigma);
}

cudaError_t launch_forward(const SceneImpl& sc, float* tau, cudaStream_t st) {
  const Geometry& g = sc.g;
  cudaError_t e = cudaMemsetAsync(tau, 0, sizeof(float) * g.S * g.B, st);
  if (e != cudaSuccess || g.P == 0 || g.S == 0) return e;

  FwdArgs a{};
  a.pairs = sc.pairs;
  a.scan = sc.scan_fwd;
  a.tau = tau;
  a.err = &sc.scratch->err;
  a.boundary = &sc.scratch->boundary_pairs;
  a.pairs_full = &sc.scratch->pairs_full;
  a.pairs_tested = &sc.scratch->pairs_tested;
  a.bounds = sc.bounds;
  a.tiles = sc.tiles;
  a.next_chunk = &sc.scratch->next_chunk;
  a.n_pairs = (uint32_t)((g.P + 1) / 2);
  a.S = (uint32_t)g.S;
  a.B = g.B;
  a.kbin = (float)((g.scan_mode == NLOS_CONFOCAL ? 2.0 : 1.0) / g.cdt);
  const bool splat = g.bin_mode == NLOS_BIN_SPLAT;
  MomTab mt{};
  const bool moments = splat && use_moments(g.sigma);
  const int mode = moments ? MODE_SPLAT_MOM
                   : splat ? MODE_SPLAT
                   : sc.params.boundary_eps > 0.f ? MODE_NEAREST_COUNT
                   : sc.occ.n > 0 ? MODE_NEAREST_OCC
                                  : MODE_NEAREST;
  if (moments) moment_table(g.sigma, mt);
  a.eps = sc.params.boundary_eps;
  if (splat) {
    const double s = g.sigma;
    a.inv2s2 = (float)(1.0 / (2.0 * s * s));
    a.norm = (float)(1.0 / (s * std::sqrt(2.0 * 3.14159265358979323846)));
    a.reach = (float)(6.0 * s);
    a.qstep = (float)std::exp(-1.0 / (s * s));
    a.R = 0;
    a.taps[0] = 1.0f;  // the flush writes the histogram unchanged
  } else {
    a.R = jitter_taps(g.sigma, a.taps, kMaxTaps);
    a.R = (a.R - 1) / 2;
    a.replicate = sc.params.jitter_padding == 1;
    if (a.replicate) jitter_tails(a.taps, a.R, a.tail);
  }

  // shared memory: histogram [bw][32] floats + two staged blocks + barriers
  int dev = sc.device, optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // pairs per staged block: NLOS_FWD_PPB, halved while the histogram of a
  // full window (up to 1024 bins) would not fit beside the two stages
  a.ppb = NLOS_FWD_PPB;
  a.stages = NLOS_FWD_STAGES;
  while (a.ppb > 256 && (size_t)std::min(g.B, 1024u) * kTile * 4 +
                                a.stages * (size_t)a.ppb * sizeof(PointPair) + 256 >
                            (size_t)optin)
    a.ppb /= 2;
  if (moments) {
    a.ppb = kPairsPerBlock;
    a.stages = 2;
  }
  // staged blocks, then full + empty barriers and the unit number of each slot
  const size_t stage_bytes = a.stages * (size_t)a.ppb * sizeof(PointPair) + 24 * a.stages + 64 +
                             8 * 32 + 4 * kRowWords;
  size_t smem;
  if (moments) {
    // window rows plus 2J halo rows fit the kMomRows moment histograms
    const uint32_t max_bw = (uint32_t)(kMomRows - 2 * mt.J) & ~3u;
    a.n_win = (g.B + max_bw - 1) / max_bw;
    a.bw = ((g.B + a.n_win - 1) / a.n_win + 3) & ~3u;
    if (a.bw > max_bw) {
      a.bw = max_bw;
      a.n_win = (g.B + a.bw - 1) / a.bw;
    }
    smem = (size_t)kMoments * kMomRows * kTile * 4 + stage_bytes;
  } else {
    uint32_t max_bw = (uint32_t)(((size_t)optin - stage_bytes) / (kTile * 4)) & ~3u;
    a.n_win = (g.B + max_bw - 1) / max_bw;
    a.bw = ((g.B + a.n_win - 1) / a.n_win + 3) & ~3u;
    smem = (size_t)a.bw * kTile * 4 + stage_bytes;
  }
  const uint32_t n_tiles = (uint32_t)((g.S + kTile - 1) / kTile);
  a.n_blk = (a.n_pairs + a.ppb - 1) / a.ppb;
  a.units = (unsigned long long)n_tiles * a.n_win * a.n_blk;

  FwdFn fn = pick(g.scan_mode, g.cos_mode, mode);
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // 1024 threads when only one CTA fits on an SM, else 512 (register budget)
  int threads = 512, per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm <= 1 || NLOS_FWD_ONE_CTA) {
    threads = 1024;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess) return e;
  }
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  unsigned long long grid = (unsigned long long)sc.num_sms * per_sm;
  if (grid > a.units) grid = a.units;
  // chunks of units claimed by the CTAs: about NLOS_FWD_CHUNKS_PER_CTA per
  // CTA, but at least 8 units (a chunk mostly ends in a tile change, whose
  // flush is worth amortising) and at most 64 (finer claims even out the
  // cost of units, which the bounds do not predict), and never so large that
  // some CTA would get none. Measured on the union (32768 units: 8 beats
  // 6.7 per chunk) and heightfield (524288 units: 64 beats 108) workloads.
  const unsigned long long per_cta = a.units / (grid * NLOS_FWD_CHUNKS_PER_CTA);
  a.chunk = std::min<unsigned long long>(std::min<unsigned long long>(std::max<unsigned long long>(per_cta, 8), 64),
                                         std::max<unsigned long long>(1, a.units / grid));
  // With block bounds, a first kernel lists the live units and the forward
  // claims chunks of that list: a chunk then holds NLOS_FWD_LIST_MIN.. units
  // that all carry work (mostly of one tile), instead of a fixed run of
  // units of which most may be culled, so tile changes (flush, zeroing,
  // barriers) are fewer per unit of work.
  ListFn lf = (NLOS_FWD_CULL && a.bounds) ? pick_list(g.scan_mode, g.cos_mode, mode) : nullptr;
  unsigned long long* list = nullptr;
  if (lf) {
    // halves (for the list kernel and the forward): two sub-blocks a unit,
    // and unit numbers that leave bits 30-31 of a list entry free
    a.list_halves = (NLOS_FWD_LIST_HALVES && a.ppb == 2 * kSubPairs &&
                     a.units < (1ull << kListHalfShift))
                        ? 1u : 0u;
    e = cudaMallocAsync(reinterpret_cast<void**>(&list), sizeof(unsigned long long) * a.units, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&sc.scratch->n_live, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
      lf<<<(unsigned)(a.units / a.n_blk), 256, 0, st>>>(a, moments ? mt.J : 0, list,
                                                          &sc.scratch->n_live);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      cudaFreeAsync(list, st);
      return e;
    }
    a.unit_list = list;
    a.n_live = &sc.scratch->n_live;
    a.list_chunks_per_cta = NLOS_FWD_LIST_CHUNKS_PER_CTA;
    a.list_min_chunk = NLOS_FWD_LIST_MIN;
    a.list_max_chunk = NLOS_FWD_LIST_MAX;
    a.list_static_pct = NLOS_FWD_LIST_STATIC;
  }
  fn<<<(unsigned)grid, threads, smem, st>>>(a, mt, sc.occ);
  e = cudaGetLastError();
  if (list) {
    const cudaError_t ef = cudaFreeAsync(list, st);
    if (e == cudaSuccess) e = ef;
  }
  return e;
}

cudaError_t launch_pair_table(const SceneImpl& sc, uint64_t s_begin, uint64_t s_count, float* u,
                              float* w, cudaStream_t st) {
  const Geometry& g = sc.g;
  const uint32_t n_pairs = (uint32_t)((g.P + 1) / 2);
  const uint64_t total = s_count * n_pairs;
  if (total == 0) return cudaSuccess;
  const float kbin = (float)((g.scan_mode == NLOS_CONFOCAL ? 2.0 : 1.0) / g.cdt);
  const unsigned blocks = (unsigned)((total + 255) / 256);
  PairTableArgs t{sc.raw_points, &sc.scratch->err, n_pairs, (uint32_t)g.P, g.scan_mode,
                  g.cos_mode, pack_const(sc.params.laser_x, sc.params.laser_y, 1.0 / g.cdt)};
#define NLOS_PT(SC, CO) \
  pair_table_kernel<SC, CO><<<blocks, 256, 0, st>>>(t, sc.scan, s_begin, s_count, kbin, u, w)
  if (g.scan_mode == NLOS_CONFOCAL) {
    if (g.cos_mode == NLOS_COS_NONE) NLOS_PT(NLOS_CONFOCAL, NLOS_COS_NONE);
    else if (g.cos_mode == NLOS_COS_OBJECT) NLOS_PT(NLOS_CONFOCAL, NLOS_COS_OBJECT);
    else NLOS_PT(NLOS_CONFOCAL, NLOS_COS_OBJECT_WALL);
  } else {
    if (g.cos_mode == NLOS_COS_NONE) NLOS_PT(NLOS_NONCONFOCAL, NLOS_COS_NONE);
    else if (g.cos_mode == NLOS_COS_OBJECT) NLOS_PT(NLOS_NONCONFOCAL, NLOS_COS_OBJECT);
    else NLOS_PT(NLOS_NONCONFOCAL, NLOS_COS_OBJECT_WALL);
  }
#undef NLOS_PT
  return cudaGetLastError();
}

}  // namespace nlos
