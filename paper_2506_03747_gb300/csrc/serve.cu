// Serving: continuous batching of simulation requests on one GB300.
//
// Host side (C++): requests are queued by nlos_serve_submit; a scheduler
// thread admits them first-in first-out while the device memory they hold
// stays within the HBM budget, uploads their points and scan tables on a copy
// stream, and publishes their work as items in a ring in mapped host memory:
//   BOX, CELL, SCAN, SCATTER  the spatial ordering of the points (a counting
//           sort by Morton cell: bounding box, cells and counts, prefix sum,
//           permutation), the same steps as the standalone scene's ordering,
//   PREP    pack the points in that order (ingest step) with the block
//           bounds, and zero the output cube,
//   FORWARD pair-histogram units (scan tile, bin window, point block) with the
//           fused jitter, exactly as the standalone forward kernel runs them,
//   REDUCE  per-cube maximum and FP64 sums,
//   NOISE   Philox/Poisson counts.
// The next phase of a request is published when the device reports the
// current one complete. Requests admitted while others run are interleaved
// item by item on the device. FORWARD items go to the main ring; the short
// items of the other phases go to an express ring, which the device drains
// first, so a request's small phases wait for at most about one running item
// per SM instead of queueing behind the forward work published before them.
//
// Device side: one persistent kernel (one CTA per SM) claims items in order
// from a device-side head counter per ring once the host has published them
// (tails in mapped memory), copies the item and its job descriptor into
// shared memory, runs it and bumps the job's phase counter in mapped memory. Every wait is
// bounded: an unpublished claimed item gives up after about a second and sets
// an error word; an idle CTA exits after the host parks the queue (or after
// about a second with nothing to do), and the host relaunches the kernel when
// new work arrives. CTAs never wait for one another.
#include "common.cuh"
#include "device_util.cuh"
#include "forward_core.cuh"
#include "noise_core.cuh"
#include "order_core.cuh"
#include "pack_core.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>
#ifdef __linux__
#include <sys/prctl.h>
#endif

namespace nlos {

nlos_status resolve_params(const nlos_params& p, uint64_t num_points, Geometry& g);
void scan_points_host(const nlos_params& p, const Geometry& g, std::vector<ScanPoint>& out);

namespace serve {

enum ItemKind : uint32_t {
  K_BOX = 0, K_CELL = 1, K_SCAN = 2, K_SCATTER = 3, K_PACK = 4, K_ZERO = 5, K_FWD = 6,
  K_REDUCE = 7, K_NOISE = 8
};
enum Phase : int {
  PH_BOX = 0, PH_CELL = 1, PH_SCAN = 2, PH_SCATTER = 3, PH_PREP = 4, PH_FWD = 5, PH_REDUCE = 6,
  PH_NOISE = 7
};
constexpr int kPhases = 8;
__host__ __device__ inline int phase_of(uint32_t kind) {
  return kind <= K_SCATTER ? (int)kind : kind <= K_ZERO ? PH_PREP : (int)kind - 1;
}

constexpr uint64_t kRing = 1ull << 16;      // work-item slots per ring (main, express)
constexpr int kMaxJobs = 1024;               // concurrently admitted requests
#ifndef NLOS_SERVE_FWD_INLINE
#define NLOS_SERVE_FWD_INLINE __forceinline__
#endif
#ifndef NLOS_SERVE_CAPBW
#define NLOS_SERVE_CAPBW 1024
#endif
#ifndef NLOS_SERVE_PPB
#define NLOS_SERVE_PPB 512
#endif
constexpr uint32_t kCapBw = NLOS_SERVE_CAPBW;  // histogram bins per window in the serving kernel
constexpr uint32_t kServePpb = NLOS_SERVE_PPB; // pairs per staged point block
constexpr uint32_t kPackChunk = 2048;        // pairs per PACK item (a multiple of kSubPairs)
static_assert(kPackChunk % kSubPairs == 0, "pack items start on sub-block edges");
constexpr uint64_t kZeroChunk = 1ull << 16;  // floats per ZERO item
constexpr uint64_t kOrderChunk = 1ull << 13; // points per BOX / CELL / SCATTER item
// FORWARD: a request's units are split into about kFwdChunksPerSm chunks per
// SM (as the standalone launch splits them), at most kFwdMaxChunk units each;
// each FORWARD item claims chunks from the request's counter, one at a time,
// so that CTAs meeting cheap (culled) units take more of them, and a CTA
// keeps its histogram across the units of one (tile, window) of a chunk. An
// item makes up to kFwdItemUnits / chunk claims (at least one): items of
// about 128 units (32 scan points x 1024 points each; at most about 1 ms)
// bound how long a new request's items wait for CTAs when every CTA has just
// started a FORWARD item, while keeping the pipeline drain and the claim at
// the end of each item rare (on a replayed mixed trace 256 units gave a
// higher median latency, four fixed claims a higher mean). Work stays
// balanced at chunk granularity: an item ends early once the counter is
// exhausted.
constexpr uint64_t kFwdChunksPerSm = 32;
constexpr uint64_t kFwdMaxChunk = 128;
constexpr uint64_t kFwdItemUnits = 128;
constexpr uint64_t kWindowPerSm = 16;        // main-ring items outstanding per SM (publication window)
constexpr uint64_t kXWindowPerSm = 32;       // express-ring items outstanding per SM
constexpr uint64_t kReduceChunk = 64;        // transients per REDUCE item
constexpr uint64_t kNoiseChunk = 1ull << 13; // bins per NOISE item
constexpr long long kIdleCycles = 2000000000LL;  // ~1 s without work: exit
constexpr long long kXtailCycles = 40000;        // ~20 us: express tail refresh while busy
constexpr int kServeThreads = 1024;           // 1 producer + 31 consumer warps (as the forward)
constexpr int kServeStages = 3;               // staged point blocks in flight
constexpr uint64_t kNone = ~0ull;
constexpr uint64_t kSkip = ~0ull - 1;

struct __align__(16) JobDesc {
  FwdArgs fwd;               // forward arguments (tau, pairs, scan, taps, ...)
  const float* raw;          // [P][8] uploaded points (submission order)
  uint32_t* perm;            // [P] packed position -> point (ordering result)
  uint16_t* cell;            // [P] Morton cell of each point
  uint32_t* cells;           // [kOrderCells] counts / cursors, then the box words
  uint32_t* counts;          // [S][B] or null
  SceneScratch* scratch;     // device
  uint64_t P, S, n;          // points, scan points, bins in the cube
  int scan_mode, cos_mode, bin_mode, noise_mode;
  PackConst pc;
  float peak_photons, dark, nr_db, pad0;
  uint64_t seed;
  uint32_t tag, pad1, pad2, pad3;
};
static_assert(sizeof(JobDesc) % 16 == 0, "JobDesc copies as int4");

struct __align__(32) WorkItem {
  uint16_t job;   // slot of the request
  uint16_t kind;
  uint32_t gen;   // the request's ticket (low bits): tells slot reuses apart
  uint64_t begin, end;
  uint64_t seq;  // == ring index once the slot is published
};
static_assert(sizeof(WorkItem) == 32, "work item layout");

struct Control {
  uint64_t tail[2];       // items published per ring (host): main, express
  uint64_t completed[2];  // items finished or skipped per ring (device)
  uint64_t err_item;   // ring index of an item whose publication wait gave up
  uint32_t park;       // host: idle CTAs may exit
  uint32_t err;        // device: kErr* bits
  int32_t alive;       // device: CTAs running
  uint32_t pad[3];
  // device: SM cycles (summed over CTAs) spent waiting for or claiming work,
  // running FORWARD items, and running the other items
  unsigned long long cycles[3];
  unsigned long long pad2;
};

struct JobStatus {
  uint32_t done[kPhases];  // items finished per phase
};

struct ServeArgs {
  Control* ctl;        // mapped
  WorkItem* ring;      // mapped [2][kRing]: main, express
  JobDesc* jobs;       // mapped [kMaxJobs]
  JobStatus* status;   // mapped [kMaxJobs]
  unsigned long long* head;  // device [2]: next index to claim per ring
};

__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

// One instance per (scan, cosine, bin mode).
template <int SCAN, int COS, int MODE>
__device__ NLOS_SERVE_FWD_INLINE bool fwd_item_mode(const FwdArgs& a, const FwdSmem& sm,
                                                    uint32_t& it, uint32_t claims) {
  FwdCount cnt;
  // whole-window flushes: row tracking costs this kernel spills, which made
  // large requests' forward items slower than the flush work it saves
  const bool ok = fwd_run_ws<SCAN, COS, MODE, 4, false>(a, 0, 0, sm, kServeStages, cnt, nullptr,
                                                     it, a.next_chunk, a.chunk, a.units,
                                                     claims);
  if ((threadIdx.x & 31) == 0 && cnt.full) atomicAdd(a.pairs_full, cnt.full * 64ull);
  if ((threadIdx.x & 31) == 0 && cnt.tested) atomicAdd(a.pairs_tested, cnt.tested * 64ull);
  return ok;
}

template <int SCAN, int COS>
__device__ bool fwd_item_cos(const FwdArgs& a, const FwdSmem& sm, uint32_t& it, int bin_mode,
                             uint32_t cl) {
  return bin_mode == NLOS_BIN_SPLAT ? fwd_item_mode<SCAN, COS, MODE_SPLAT>(a, sm, it, cl)
                                    : fwd_item_mode<SCAN, COS, MODE_NEAREST>(a, sm, it, cl);
}

// FORWARD: up to `cl` chunks of the job's units (the item's `end`), claimed
// from its counter.
__device__ bool fwd_item(const JobDesc& j, const FwdSmem& sm, uint32_t& it, uint32_t cl) {
  const FwdArgs& a = j.fwd;
  const int m = j.bin_mode;
  if (j.scan_mode == NLOS_CONFOCAL) {
    if (j.cos_mode == NLOS_COS_NONE) return fwd_item_cos<NLOS_CONFOCAL, NLOS_COS_NONE>(a, sm, it, m, cl);
    if (j.cos_mode == NLOS_COS_OBJECT) return fwd_item_cos<NLOS_CONFOCAL, NLOS_COS_OBJECT>(a, sm, it, m, cl);
    return fwd_item_cos<NLOS_CONFOCAL, NLOS_COS_OBJECT_WALL>(a, sm, it, m, cl);
  }
  if (j.cos_mode == NLOS_COS_NONE) return fwd_item_cos<NLOS_NONCONFOCAL, NLOS_COS_NONE>(a, sm, it, m, cl);
  if (j.cos_mode == NLOS_COS_OBJECT) return fwd_item_cos<NLOS_NONCONFOCAL, NLOS_COS_OBJECT>(a, sm, it, m, cl);
  return fwd_item_cos<NLOS_NONCONFOCAL, NLOS_COS_OBJECT_WALL>(a, sm, it, m, cl);
}

// REDUCE: transients [b, e) of the job, one warp per transient; the cube's
// maximum and FP64 sums go to the job's scratch, one atomic per item and
// quantity (same-address atomics from every warp would serialise). red:
// shared scratch of 3 doubles per warp.
__device__ __noinline__ void reduce_item(const JobDesc& j, uint64_t b, uint64_t e, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t B = j.fwd.B;
  double csum = 0.0, csq = 0.0;
  float cmax = 0.0f;
  for (uint64_t t = b + warp; t < e; t += nwarps) {
    const float* row = j.fwd.tau + t * B;
    double s = 0.0, q = 0.0;
    float m = 0.0f;
    for (uint32_t i = lane; i < B; i += 32) {
      const float v = row[i];
      s += (double)v;
      q += (double)v * v;
      m = fmaxf(m, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      q += __shfl_xor_sync(0xffffffffu, q, o);
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    csum += s;
    csq += q;
    cmax = fmaxf(cmax, m);
  }
  if (lane == 0) {
    red[warp] = csum;
    red[nwarps + warp] = csq;
    red[2 * nwarps + warp] = (double)cmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, q = 0.0, m = 0.0;
    for (int w = 0; w < nwarps; ++w) {
      s += red[w];
      q += red[nwarps + w];
      m = fmax(m, red[2 * nwarps + w]);
    }
    atomicMax(&j.scratch->peak_bits, __float_as_uint((float)m));
    atomicAdd(&j.scratch->sum, s);
    atomicAdd(&j.scratch->sumsq, q);
  }
}

// NOISE: bins [b, e) of the job; scale from the job's reduction.
__device__ __noinline__ void noise_item(const JobDesc& j, uint64_t b, uint64_t e) {
  const float scale = noise_scale_from(j.scratch, j.noise_mode, j.peak_photons, j.nr_db, j.n);
  if (b == 0 && threadIdx.x == 0) {
    j.scratch->scale = scale;
    j.scratch->dark = j.dark;
  }
  // groups of four bins (one Philox block for their first draws); a group
  // that straddles an item edge is drawn by both items, each keeping its bins
  noise_groups(j.fwd.tau, j.counts, b, e, 0, scale, j.dark, j.seed, j.tag, nullptr, threadIdx.x,
               blockDim.x);
}

// PACK: pairs [b, e) of the job (each item kind runs in its own frame, so
// the pack's registers do not weigh on the forward's)
__device__ __noinline__ void pack_item(const JobDesc& j, uint64_t b, uint64_t e) {
  for (uint64_t k = b + threadIdx.x; k < e; k += blockDim.x)
    pack_pair(j.raw, j.P, k, j.scan_mode, j.cos_mode, j.pc,
              const_cast<PointPair*>(j.fwd.pairs), &j.scratch->err, j.perm);
  // bounds of the sub-blocks this item packs (items start on sub-block edges)
  const uint64_t sb_end = (e + kSubPairs - 1) / kSubPairs;
  for (uint64_t sb = b / kSubPairs + (threadIdx.x >> 5); sb < sb_end; sb += blockDim.x >> 5)
    block_bound_warp(j.raw, j.P, sb, j.scan_mode, j.cos_mode, j.pc, j.perm,
                     const_cast<BlockBound*>(j.fwd.bounds) + sb);
}

// full[i] (one arrival: the producer's expect_tx) and empty[i] (one arrival
// per consumer warp) for each stage.
__device__ void init_stage_barriers(uint64_t* bars) {
  for (int i = 0; i < kServeStages; ++i) {
    mbar_init(&bars[i], 1);
    mbar_init(&bars[kServeStages + i], kServeThreads / 32 - 1);
  }
  fence_mbar_init();
}

__global__ void __launch_bounds__(kServeThreads, 1) serve_kernel(const ServeArgs q) {
  extern __shared__ __align__(128) unsigned char smem[];
  FwdSmem sm;
  sm.hist = reinterpret_cast<float*>(smem);
  sm.stage = reinterpret_cast<PointPair*>(smem + (size_t)kCapBw * kTile * 4);
  sm.bars = reinterpret_cast<uint64_t*>(sm.stage + kServeStages * kServePpb);
  sm.units = reinterpret_cast<unsigned long long*>(sm.bars + 2 * kServeStages);
  JobDesc* jd = reinterpret_cast<JobDesc*>(sm.units + kServeStages + 1);
  __shared__ WorkItem s_item;
  __shared__ unsigned long long s_idx;
  __shared__ int s_lane;  // ring of the claimed item
  // State that thread 0 alone uses, and the descriptor cache, in shared
  // memory: kept in registers it would be live in every thread across the
  // forward items, whose unrolled loop needs all 64.
  struct LoopState {
    unsigned long long tail_seen;  // last main-ring tail read from host memory
    unsigned long long xtail_seen; // last express-ring tail read from host memory
    long long xtail_time;          // when it was read
    unsigned long long cyc[3];     // waiting, FORWARD items, other items
    long long t_mark;
    uint32_t cached_job, cached_gen;
  };
  __shared__ LoopState st;

  const int tid = threadIdx.x;
  if (tid == 0) {
    init_stage_barriers(sm.bars);
    atomicAdd_system(&q.ctl->alive, 1);
    st.tail_seen = 0;
    st.xtail_seen = 0;
    st.xtail_time = 0;
    st.cyc[0] = st.cyc[1] = st.cyc[2] = 0;
    st.t_mark = clock64();
    st.cached_job = 0xFFFFFFFFu;
    st.cached_gen = 0;
  }
  __syncthreads();
  uint32_t it = 0;

  for (;;) {
    if (tid == 0) {
      // claim the next published index: express ring first, then the main
      // ring, each by compare-and-swap on its device head against a cached
      // copy of its tail (tails only grow, so a stale value is a safe
      // bound). The main tail is read again from host memory when the head
      // has caught up with the cached value; the express tail on every pass
      // while the main ring looks empty, else at most every kXtailCycles (so
      // that 152 CTAs claiming short FORWARD items do not all read the same
      // host cache line on every claim, which starved them)
      unsigned long long got = kNone;
      int lane = 0;
      const long long t0 = clock64();
      unsigned long long h = *reinterpret_cast<volatile unsigned long long*>(q.head);
      for (;;) {
        const long long tnow = clock64();
        if (!(h < st.tail_seen) || tnow - st.xtail_time > kXtailCycles) {
          st.xtail_seen = ld_acquire_sys(&q.ctl->tail[1]);
          st.xtail_time = tnow;
        }
        const unsigned long long xt = st.xtail_seen;
        unsigned long long xh = *reinterpret_cast<volatile unsigned long long*>(q.head + 1);
        while (xh < xt) {
          const unsigned long long seen = atomicCAS(q.head + 1, xh, xh + 1);
          if (seen == xh) {
            got = xh;
            lane = 1;
            break;
          }
          xh = seen;
        }
        if (got != kNone) break;
        if (h < st.tail_seen) {
          const unsigned long long seen = atomicCAS(q.head, h, h + 1);
          if (seen == h) {
            got = h;
            break;
          }
          h = seen;  // another CTA moved the head: retry from there
          continue;
        }
        st.tail_seen = ld_acquire_sys(&q.ctl->tail[0]);
        if (h < st.tail_seen) continue;
        if (ld_volatile_u32(&q.ctl->park)) break;
        if (clock64() - t0 > kIdleCycles) break;
        __nanosleep(500);
        h = *reinterpret_cast<volatile unsigned long long*>(q.head);
      }
      if (got != kNone) {
        // the slot is written before the tail moves; a withheld publication
        // leaves a stale sequence number: wait (bounded), then give up
        WorkItem* slot = q.ring + (uint64_t)lane * kRing + (got % kRing);
        const long long t1 = clock64();
        while (ld_acquire_sys(&slot->seq) != got) {
          if (clock64() - t1 > kWaitCycles) {
            *reinterpret_cast<volatile uint64_t*>(&q.ctl->err_item) = got;
            __threadfence_system();
            atomicOr_system(&q.ctl->err, kErrWaitTimeout);
            got = kSkip;
            break;
          }
          __nanosleep(200);
        }
        if (got != kSkip) s_item = *slot;
      }
      s_idx = got;
      s_lane = lane;
      const long long now = clock64();
      st.cyc[0] += (unsigned long long)(now - st.t_mark);
      st.t_mark = now;
    }
    __syncthreads();
    const unsigned long long idx = s_idx;
    if (idx == kNone) break;
    if (idx == kSkip) {
      if (tid == 0) {
        __threadfence_system();
        atomicAdd_system(reinterpret_cast<unsigned long long*>(&q.ctl->completed[s_lane]), 1ull);
      }
      __syncthreads();
      continue;
    }
    // the item is read from shared memory where it is used (s_item changes
    // only at the next claim, after the barrier that ends this item)
    const WorkItem& item = s_item;
    // job descriptor: mapped memory -> shared memory, unless this CTA holds
    // it already (consecutive items mostly belong to one request; a slot's
    // descriptor only changes with a new request, i.e. a new gen). Every
    // thread reads the cache tags before thread 0 updates them, after the
    // barrier.
    if (item.job != st.cached_job || item.gen != st.cached_gen) {
      const int4* src = reinterpret_cast<const int4*>(q.jobs + item.job);
      int4* dst = reinterpret_cast<int4*>(jd);
      for (int i = tid; i < (int)(sizeof(JobDesc) / 16); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      if (tid == 0) {
        st.cached_job = item.job;
        st.cached_gen = item.gen;
      }
    }
    switch (item.kind) {
      case K_BOX:  // the histogram's shared memory is free between forward items
        // the first item also zeroes the cell counts (CELL items start only
        // once every BOX item has finished)
        if (item.begin == 0)
          for (uint32_t k = tid; k < kOrderCells; k += blockDim.x) jd->cells[k] = 0u;
        box_range(jd->raw, item.begin, item.end, tid, blockDim.x, jd->cells + kOrderCells,
                  reinterpret_cast<uint32_t*>(sm.hist));
        break;
      case K_CELL:
        cell_range(jd->raw, item.begin, item.end, tid, blockDim.x, jd->cells + kOrderCells,
                   jd->cell, jd->cells);
        break;
      case K_SCAN:
        scan_cells(jd->cells, reinterpret_cast<uint32_t*>(sm.hist));
        break;
      case K_SCATTER:
        scatter_range(jd->cell, item.begin, item.end, tid, blockDim.x, jd->cells, jd->perm);
        break;
      case K_PACK:
        pack_item(*jd, item.begin, item.end);
        break;
      case K_ZERO:
        for (uint64_t k = item.begin + tid; k < item.end; k += blockDim.x) jd->fwd.tau[k] = 0.0f;
        break;
      case K_FWD:
        // a forward wait that gave up is recorded in the job error word; the
        // stage barriers are then out of step with the unit counter: start
        // them afresh (every copy has landed or been waited for, bounded)
        if (!fwd_item(*jd, sm, it, (uint32_t)item.end)) {
          if (tid == 0) {
            for (int i = 0; i < 2 * kServeStages; ++i) mbar_inval(&sm.bars[i]);
            init_stage_barriers(sm.bars);
          }
          it = 0;
        }
        break;
      case K_REDUCE:
        reduce_item(*jd, item.begin, item.end, reinterpret_cast<double*>(sm.hist));
        break;
      default:
        noise_item(*jd, item.begin, item.end);
        break;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence_system();
      atomicAdd_system(&q.status[item.job].done[phase_of(item.kind)], 1u);
      atomicAdd_system(reinterpret_cast<unsigned long long*>(&q.ctl->completed[s_lane]), 1ull);
      const long long now = clock64();
      st.cyc[item.kind == K_FWD ? 1 : 2] += (unsigned long long)(now - st.t_mark);
      st.t_mark = now;
    }
  }
  if (tid == 0) {
    st.cyc[0] += (unsigned long long)(clock64() - st.t_mark);
    for (int k = 0; k < 3; ++k) atomicAdd_system(&q.ctl->cycles[k], st.cyc[k]);
    atomicSub_system(&q.ctl->alive, 1);
  }
}

// ---------------------------------------------------------------------------
// Host scheduler.
// ---------------------------------------------------------------------------
using Clock = std::chrono::steady_clock;

enum ReqState { R_PENDING, R_UPLOAD, R_RUNNING, R_DRAINING, R_FINISHING, R_DONE, R_FAILED, R_CANCELLED };

struct Request {
  uint64_t ticket = 0;
  nlos_params params{};
  Geometry g{};
  std::vector<float> pts;
  ReqState state = R_PENDING;
  nlos_status status = NLOS_OK;
  std::string msg;
  int slot = -1;
  char* dev = nullptr;
  size_t bytes = 0;
  PointPair* pairs = nullptr;
  float* raw = nullptr;
  uint32_t* perm = nullptr;
  uint16_t* cell = nullptr;
  uint32_t* cells = nullptr;
  ScanPoint* scan = nullptr;
  float* tau = nullptr;
  uint32_t* counts = nullptr;
  SceneScratch* scratch = nullptr;
  BlockBound* bounds = nullptr;
  TileBound* tiles = nullptr;
  SceneScratch* h_scratch = nullptr;  // pinned copy at completion (the slot's pool entry)
  cudaEvent_t ev = nullptr;
  std::atomic<int> upload{0};  // 0 queued, 1 copies issued (ev recorded), 2 failed
  std::string upload_msg;
  int phase = 0;
  uint32_t items[kPhases] = {};
  uint32_t withheld = 0;  // published items that will never complete (fault injection)
  std::vector<WorkItem> backlog;  // items of the current phase not yet published
  size_t backlog_pos = 0;
  bool release_on_done = false;
  Clock::time_point t_submit, t_done;
  Clock::time_point t_mark[2 + kPhases];  // tracing: admit, upload done, each phase done
  uint32_t items_total = 0;
  nlos_stats stats{};
};

struct Server {
  uint64_t budget = 0, resident = 0;
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<Request*> active;
  std::vector<int> free_slots;
  std::thread th;
  std::atomic<bool> stop{false};
  // uploads run on their own thread: a copy from pageable memory returns only
  // once the data is staged, and must not hold up the scheduler
  std::vector<std::thread> uploaders;
  std::mutex upmu;
  std::condition_variable upcv;
  std::deque<Request*> upq;
  uint64_t next_ticket = 1;
  int device = 0, num_sms = 0;
  cudaStream_t kstream = nullptr, cstream = nullptr;
  Control* ctl = nullptr;       // host addresses of the mapped structures
  WorkItem* ring = nullptr;
  JobDesc* jobs = nullptr;
  JobStatus* status = nullptr;
  // pinned per-slot copies of the request scratch at completion; allocated
  // once, because cudaFreeHost waits for all device work (the persistent
  // kernel included) and cudaHostAlloc may synchronise too
  SceneScratch* h_scratch = nullptr;
  ServeArgs dev_args{};         // device addresses of the same memory
  unsigned long long* d_head = nullptr;  // [2]
  uint64_t published[2] = {0, 0};       // per ring: main, express
  uint64_t window[2] = {0, 0};          // items outstanding on the device at most, per ring
  std::vector<std::pair<double, Request*>> fwd_order;  // publish_window's scratch
  bool kernel_running = false;
  cudaEvent_t kernel_done = nullptr;
  size_t smem = 0;
  FILE* trace = nullptr;  // NLOS_SERVE_TRACE
  // fault injection (tests)
  int inject = 0;
  uint64_t withheld_item = kNone;
  Request* withheld_req = nullptr;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

void carve(Request* r) {
  const Geometry& g = r->g;
  const uint64_t n_pairs = (g.P + 1) / 2;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  size_t o_pairs = take(sizeof(PointPair) * (n_pairs ? n_pairs : 1));
  size_t o_raw = take(sizeof(float) * 8 * (g.P ? g.P : 1));
  size_t o_perm = take(sizeof(uint32_t) * (g.P ? g.P : 1));
  size_t o_cell = take(sizeof(uint16_t) * (g.P ? g.P : 1));
  size_t o_cells = take(sizeof(uint32_t) * (kOrderCells + kOrderBoxWords));
  size_t o_scan = take(sizeof(ScanPoint) * g.S);
  size_t o_tau = take(sizeof(float) * g.S * g.B);
  size_t o_cnt = g.noise_mode != NLOS_NOISE_NONE ? take(sizeof(uint32_t) * g.S * g.B) : 0;
  size_t o_scr = take(sizeof(SceneScratch));
  const uint64_t n_sub = (n_pairs + kSubPairs - 1) / kSubPairs;
  size_t o_bnd = take(sizeof(BlockBound) * (n_sub ? n_sub : 1));
  size_t o_til = take(sizeof(TileBound) * ((g.S + kTile - 1) / kTile));
  r->bytes = off;
  if (!r->dev) return;
  r->pairs = reinterpret_cast<PointPair*>(r->dev + o_pairs);
  r->raw = reinterpret_cast<float*>(r->dev + o_raw);
  r->perm = reinterpret_cast<uint32_t*>(r->dev + o_perm);
  r->cell = reinterpret_cast<uint16_t*>(r->dev + o_cell);
  r->cells = reinterpret_cast<uint32_t*>(r->dev + o_cells);
  r->scan = reinterpret_cast<ScanPoint*>(r->dev + o_scan);
  r->tau = reinterpret_cast<float*>(r->dev + o_tau);
  r->counts = g.noise_mode != NLOS_NOISE_NONE ? reinterpret_cast<uint32_t*>(r->dev + o_cnt) : nullptr;
  r->scratch = reinterpret_cast<SceneScratch*>(r->dev + o_scr);
  r->bounds = reinterpret_cast<BlockBound*>(r->dev + o_bnd);
  r->tiles = reinterpret_cast<TileBound*>(r->dev + o_til);
}

void fill_job(Server& sv, Request* r, JobDesc& j) {
  std::memset(&j, 0, sizeof(j));
  const Geometry& g = r->g;
  const nlos_params& p = r->params;
  FwdArgs& a = j.fwd;
  a.pairs = r->pairs;
  a.scan = r->scan;
  a.tau = r->tau;
  a.err = &r->scratch->err;
  a.boundary = &r->scratch->boundary_pairs;
  a.pairs_full = &r->scratch->pairs_full;
  a.pairs_tested = &r->scratch->pairs_tested;
  a.bounds = r->bounds;
  a.tiles = r->tiles;
  a.n_pairs = (uint32_t)((g.P + 1) / 2);
  a.S = (uint32_t)g.S;
  a.B = g.B;
  a.kbin = (float)((g.scan_mode == NLOS_CONFOCAL ? 2.0 : 1.0) / g.cdt);
  a.ppb = kServePpb;
  a.stages = kServeStages;
  a.n_win = (g.B + kCapBw - 1) / kCapBw;
  a.bw = ((g.B + a.n_win - 1) / a.n_win + 3) & ~3u;
  a.n_blk = (a.n_pairs + a.ppb - 1) / a.ppb;
  a.units = (unsigned long long)((g.S + kTile - 1) / kTile) * a.n_win * a.n_blk;
  a.next_chunk = &r->scratch->next_chunk;  // zero from the upload
  a.chunk = std::min<unsigned long long>(
      kFwdMaxChunk, std::max<unsigned long long>(1, a.units / ((uint64_t)sv.num_sms * kFwdChunksPerSm)));
  a.replicate = 0;
  if (g.bin_mode == NLOS_BIN_SPLAT) {
    const double s = g.sigma;
    a.inv2s2 = (float)(1.0 / (2.0 * s * s));
    a.norm = (float)(1.0 / (s * std::sqrt(2.0 * 3.14159265358979323846)));
    a.reach = (float)(6.0 * s);
    a.qstep = (float)std::exp(-1.0 / (s * s));
    a.R = 0;
    a.taps[0] = 1.0f;
  } else {
    a.R = (jitter_taps(g.sigma, a.taps, kMaxTaps) - 1) / 2;
    a.replicate = r->params.jitter_padding == 1;
    if (a.replicate) jitter_tails(a.taps, a.R, a.tail);
  }
  j.raw = r->raw;
  j.perm = r->perm;
  j.cell = r->cell;
  j.cells = r->cells;
  j.counts = r->counts;
  j.scratch = r->scratch;
  j.P = g.P;
  j.S = g.S;
  j.n = g.S * (uint64_t)g.B;
  j.scan_mode = g.scan_mode;
  j.cos_mode = g.cos_mode;
  j.bin_mode = g.bin_mode;
  j.noise_mode = g.noise_mode;
  j.pc = pack_const(p.laser_x, p.laser_y, 1.0 / g.cdt);
  j.peak_photons = p.peak_photons;
  j.dark = p.dark_per_bin;
  j.nr_db = p.nr_db;
  j.seed = p.seed;
  j.tag = p.stream_tag;
}

// The ring a phase's items go to: FORWARD to the main ring, the rest to the
// express ring.
int lane_of(int phase) { return phase == PH_FWD ? 0 : 1; }

// Writes up to max_items backlog items of r into the ring of its phase and
// moves that ring's tail (release); returns how many it wrote.
size_t publish_some(Server& sv, Request* r, size_t max_items) {
  const size_t n = std::min(max_items, r->backlog.size() - r->backlog_pos);
  if (n == 0) return 0;
  const int lane = lane_of(r->phase);
  uint64_t idx = sv.published[lane];
  for (size_t k = 0; k < n; ++k) {
    const WorkItem& w = r->backlog[r->backlog_pos + k];
    WorkItem* slot = sv.ring + (uint64_t)lane * kRing + (idx % kRing);
    slot->job = w.job;
    slot->kind = w.kind;
    slot->gen = w.gen;
    slot->begin = w.begin;
    slot->end = w.end;
    if (sv.inject == 1 && sv.withheld_item == kNone) {
      // fault injection: the slot of this item is never published
      sv.withheld_item = idx;
      sv.withheld_req = r;
      r->withheld += 1;
      sv.inject = 0;
    } else {
      __atomic_store_n(&slot->seq, idx, __ATOMIC_RELEASE);
    }
    ++idx;
  }
  std::atomic_thread_fence(std::memory_order_seq_cst);
  __atomic_store_n(&sv.ctl->tail[lane], idx, __ATOMIC_RELEASE);
  r->backlog_pos += n;
  sv.published[lane] = idx;
  if (r->backlog_pos == r->backlog.size()) {
    r->backlog.clear();
    r->backlog.shrink_to_fit();
    r->backlog_pos = 0;
  }
  return n;
}

// Publishes backlog items of the running requests while fewer than the
// ring's window of items are outstanding on the device. Express items go
// oldest request first. FORWARD items: the oldest request with FORWARD work
// may keep a quarter of the window outstanding, the rest goes shortest
// remaining work first (the pairs of a request's unpublished FORWARD items).
// A small request then does not wait behind the forward of a large one
// submitted before it (which is what sets the median latency under first-in
// first-out), while the oldest request keeps at least about a quarter of the
// device, so a stream of small requests cannot starve a large one. (On a
// replayed mixed trace, a half share gave a higher median, pure shortest-
// remaining-first a longer tail, and aging by a fixed age both.) Each window (a few
// items per SM) stays far below half its ring, which the claim protocol
// requires.
void publish_window(Server& sv) {
  uint64_t outstanding[2];
  for (int l = 0; l < 2; ++l)
    outstanding[l] = sv.published[l] - __atomic_load_n(&sv.ctl->completed[l], __ATOMIC_ACQUIRE);
  std::vector<std::pair<double, Request*>>& fwd = sv.fwd_order;
  fwd.clear();
  bool oldest = true;
  for (Request* r : sv.active) {
    if (r->state != R_RUNNING || r->backlog.empty()) continue;
    const int l = lane_of(r->phase);
    if (l == 0) {
      if (oldest) {
        oldest = false;
        const uint64_t mine =
            r->backlog_pos - __atomic_load_n(&sv.status[r->slot].done[PH_FWD], __ATOMIC_ACQUIRE);
        const uint64_t share = sv.window[0] / 4;
        if (mine < share && outstanding[0] < sv.window[0])
          outstanding[0] += publish_some(
              sv, r, (size_t)std::min(share - mine, sv.window[0] - outstanding[0]));
        if (r->backlog.empty()) continue;
      }
      const double left = (double)(r->backlog.size() - r->backlog_pos) /
                          (double)std::max<uint32_t>(1, r->items[PH_FWD]);
      fwd.emplace_back(left * (double)r->g.S * (double)r->g.P, r);
    } else if (outstanding[1] < sv.window[1]) {
      outstanding[1] += publish_some(sv, r, (size_t)(sv.window[1] - outstanding[1]));
    }
  }
  std::stable_sort(fwd.begin(), fwd.end(),
                   [](const std::pair<double, Request*>& a, const std::pair<double, Request*>& b) {
                     return a.first < b.first;
                   });
  for (auto& f : fwd) {
    if (outstanding[0] >= sv.window[0]) break;
    outstanding[0] += publish_some(sv, f.second, (size_t)(sv.window[0] - outstanding[0]));
  }
}

void publish_phase(Server& sv, Request* r, int phase) {
  const Geometry& g = r->g;
  std::vector<WorkItem> items;
  const uint16_t job = (uint16_t)r->slot;
  const uint32_t gen = (uint32_t)r->ticket;
  if (phase >= PH_BOX && phase <= PH_SCATTER) {
    if (phase == PH_SCAN) {
      if (g.P) items.push_back({job, K_SCAN, gen, 0, 0, 0});
    } else {
      for (uint64_t b = 0; b < g.P; b += kOrderChunk)
        items.push_back({job, (uint16_t)phase, gen, b, std::min<uint64_t>(g.P, b + kOrderChunk), 0});
    }
  } else if (phase == PH_PREP) {
    const uint64_t n_pairs = (g.P + 1) / 2;
    for (uint64_t b = 0; b < n_pairs; b += kPackChunk)
      items.push_back({job, K_PACK, gen, b, std::min<uint64_t>(n_pairs, b + kPackChunk), 0});
    const uint64_t n = g.S * (uint64_t)g.B;
    for (uint64_t b = 0; b < n; b += kZeroChunk)
      items.push_back({job, K_ZERO, gen, b, std::min<uint64_t>(n, b + kZeroChunk), 0});
  } else if (phase == PH_FWD) {
    // enough items for every chunk to be claimed: each makes `claims`
    // claims (its `end`) unless the counter has passed the last chunk
    const FwdArgs& a = sv.jobs[job].fwd;
    const uint64_t chunks = (a.units + a.chunk - 1) / a.chunk;
    const uint64_t claims = std::max<uint64_t>(1, kFwdItemUnits / a.chunk);
    const uint64_t n_items = (chunks + claims - 1) / claims;
    for (uint64_t i = 0; i < n_items; ++i) items.push_back({job, K_FWD, gen, 0, claims, 0});
  } else if (phase == PH_REDUCE) {
    for (uint64_t b = 0; b < g.S; b += kReduceChunk)
      items.push_back({job, K_REDUCE, gen, b, std::min<uint64_t>(g.S, b + kReduceChunk), 0});
  } else {
    const uint64_t n = g.S * (uint64_t)g.B;
    for (uint64_t b = 0; b < n; b += kNoiseChunk)
      items.push_back({job, K_NOISE, gen, b, std::min<uint64_t>(n, b + kNoiseChunk), 0});
  }
  r->phase = phase;
  r->items[phase] = (uint32_t)items.size();
  r->backlog = std::move(items);
  r->backlog_pos = 0;
}

// Per-request phase timestamps (milliseconds since submission) appended as a
// JSON line to the file named by NLOS_SERVE_TRACE, if set.
void trace_request(Server& sv, Request* r) {
  if (!sv.trace) return;
  auto ms = [&](Clock::time_point t) {
    return t.time_since_epoch().count() == 0
               ? -1.0
               : std::chrono::duration<double, std::milli>(t - r->t_submit).count();
  };
  std::fprintf(sv.trace,
               "{\"ticket\": %llu, \"S\": %llu, \"B\": %u, \"P\": %llu, \"items\": %u, "
               "\"status\": %d, \"admit\": %.3f, \"uploaded\": %.3f, \"ordered\": %.3f, "
               "\"prep\": %.3f, \"forward\": %.3f, \"reduce\": %.3f, \"noise\": %.3f, "
               "\"done\": %.3f}\n",
               (unsigned long long)r->ticket, (unsigned long long)r->g.S, r->g.B,
               (unsigned long long)r->g.P, r->items_total, (int)r->status, ms(r->t_mark[0]),
               ms(r->t_mark[1]), ms(r->t_mark[2 + PH_SCATTER]), ms(r->t_mark[2 + PH_PREP]),
               ms(r->t_mark[2 + PH_FWD]), ms(r->t_mark[2 + PH_REDUCE]),
               ms(r->t_mark[2 + PH_NOISE]), ms(r->t_done));
  std::fflush(sv.trace);
}

void finish(Server& sv, Request* r, nlos_status st, const std::string& msg) {
  r->status = st;
  r->msg = msg;
  r->state = st == NLOS_OK ? R_DONE : R_FAILED;
  r->t_done = Clock::now();
  (void)sv;
}

void free_request_memory(Server& sv, Request* r) {
  if (r->dev) {
    cudaFreeAsync(r->dev, sv.cstream);
    sv.resident -= r->bytes;
    r->dev = nullptr;
  }
  if (r->slot >= 0) {
    sv.free_slots.push_back(r->slot);
    r->slot = -1;
  }
}

void destroy_request(Server& sv, Request* r) {
  free_request_memory(sv, r);
  if (r->ev) cudaEventDestroy(r->ev);
  sv.reqs.erase(r->ticket);
  delete r;
}

// One scheduler pass (called with the lock held).
bool step(Server& sv) {
  bool busy = false;
  // admission, first-in first-out within the budget
  while (!sv.pending.empty() && !sv.free_slots.empty()) {
    Request* r = sv.pending.front();
    carve(r);
    if (r->bytes > sv.budget) {
      sv.pending.pop_front();
      finish(sv, r, NLOS_ENOMEM, "request needs more device memory than the server budget");
      continue;
    }
    if (sv.resident + r->bytes > sv.budget) break;
    sv.pending.pop_front();
    if (sv.inject == 2) {
      sv.inject = 0;
      finish(sv, r, NLOS_ENOMEM, "device allocation refused (injected)");
      continue;
    }
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&r->dev), r->bytes, sv.cstream);
    if (e != cudaSuccess) {
      r->dev = nullptr;
      finish(sv, r, NLOS_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
      continue;
    }
    sv.resident += r->bytes;
    carve(r);
    r->slot = sv.free_slots.back();
    sv.free_slots.pop_back();
    r->h_scratch = sv.h_scratch + r->slot;
    std::memset(&sv.status[r->slot], 0, sizeof(JobStatus));
    // uploads on the copy stream (copy engines only: the serving kernel may be
    // occupying every SM), issued by the uploader thread
    r->upload.store(0);
    {
      std::lock_guard<std::mutex> ul(sv.upmu);
      sv.upq.push_back(r);
    }
    sv.upcv.notify_one();
    r->state = R_UPLOAD;
    r->t_mark[0] = Clock::now();
    sv.active.push_back(r);
    busy = true;
  }
  // progress of admitted requests
  const uint32_t dev_err = __atomic_load_n(&sv.ctl->err, __ATOMIC_ACQUIRE);
  for (size_t i = 0; i < sv.active.size();) {
    Request* r = sv.active[i];
    bool leave = false;
    if (r->state == R_UPLOAD) {
      const int up = r->upload.load(std::memory_order_acquire);
      if (up == 2) {
        free_request_memory(sv, r);
        finish(sv, r, NLOS_ECUDA, r->upload_msg);
        leave = true;
      } else if (up == 1 && cudaEventQuery(r->ev) == cudaSuccess) {
        r->pts.clear();
        r->pts.shrink_to_fit();
        fill_job(sv, r, sv.jobs[r->slot]);
        std::atomic_thread_fence(std::memory_order_seq_cst);
        r->state = R_RUNNING;
        r->t_mark[1] = Clock::now();
        publish_phase(sv, r, PH_BOX);
        busy = true;
      }
    } else if (r->state == R_RUNNING) {
      if (!r->backlog.empty()) busy = true;
      if (sv.withheld_req == r && (dev_err & kErrWaitTimeout)) {
        // the device gave up on the withheld item: the request cannot finish;
        // its memory stays until every other item published for it is done
        // (items not yet published never will be)
        sv.withheld_req = nullptr;
        r->withheld += (uint32_t)(r->backlog.size() - r->backlog_pos);
        r->backlog.clear();
        r->backlog_pos = 0;
        r->state = R_DRAINING;
        r->status = NLOS_ETIMEOUT;
        r->msg = "a work item was never published; the device wait gave up";
        busy = true;
      } else {
        const uint32_t done = __atomic_load_n(&sv.status[r->slot].done[r->phase], __ATOMIC_ACQUIRE);
        if (done >= r->items[r->phase]) {
          r->t_mark[2 + r->phase] = Clock::now();
          r->items_total += r->items[r->phase];
          int next = r->phase + 1;
          if (next == PH_NOISE && r->g.noise_mode == NLOS_NOISE_NONE) next = kPhases;
          if (next <= PH_NOISE) {
            publish_phase(sv, r, next);
          } else {
            cudaMemcpyAsync(r->h_scratch, r->scratch, sizeof(SceneScratch), cudaMemcpyDeviceToHost, sv.cstream);
            cudaEventRecord(r->ev, sv.cstream);
            r->state = R_FINISHING;
          }
          busy = true;
        }
      }
    } else if (r->state == R_DRAINING) {
      uint32_t done = 0, total = 0;
      for (int ph = 0; ph <= r->phase; ++ph) {
        done += __atomic_load_n(&sv.status[r->slot].done[ph], __ATOMIC_ACQUIRE);
        total += r->items[ph];
      }
      if (done + r->withheld >= total) {
        r->state = R_FAILED;
        r->t_done = Clock::now();
        leave = true;
      }
    } else if (r->state == R_FINISHING) {
      if (cudaEventQuery(r->ev) == cudaSuccess) {
        const SceneScratch& h = *r->h_scratch;
        const uint64_t n = r->g.S * (uint64_t)r->g.B;
        nlos_stats& s = r->stats;
        s.struct_size = sizeof(nlos_stats);
        s.pairs = r->g.S * r->g.P;
        float peak;
        std::memcpy(&peak, &h.peak_bits, sizeof(peak));
        s.peak = peak;
        s.mean = n ? h.sum / (double)n : 0.0;
        s.variance = n ? std::max(0.0, h.sumsq / (double)n - s.mean * s.mean) : 0.0;
        s.noise_scale = r->counts ? h.scale : 0.0;
        s.noise_dark = r->counts ? h.dark : 0.0;
        s.device_error = h.err;
        s.pairs_full = h.pairs_full;
        s.pairs_tested = h.pairs_tested;
        if (h.err & kErrBadPoint) finish(sv, r, NLOS_EINVAL, "invalid surface point");
        else if (h.err & kErrWaitTimeout) finish(sv, r, NLOS_ETIMEOUT, "a bounded device wait gave up");
        else finish(sv, r, NLOS_OK, "");
        leave = true;
      }
    }
    if (leave) {
      trace_request(sv, r);
      sv.active.erase(sv.active.begin() + i);
      if (r->status != NLOS_OK) free_request_memory(sv, r);
      if (r->release_on_done) destroy_request(sv, r);
      sv.cv_done.notify_all();
    } else {
      ++i;
    }
  }
  publish_window(sv);
  // kernel lifecycle: run while items are outstanding, park when idle
  bool outstanding = false;
  for (int l = 0; l < 2; ++l)
    outstanding |= sv.published[l] > __atomic_load_n(&sv.ctl->completed[l], __ATOMIC_ACQUIRE);
  if (sv.kernel_running && cudaEventQuery(sv.kernel_done) == cudaSuccess) sv.kernel_running = false;
  if (outstanding && !sv.kernel_running) {
    __atomic_store_n(&sv.ctl->park, 0u, __ATOMIC_RELEASE);
    ServeArgs q = sv.dev_args;
    serve_kernel<<<sv.num_sms, kServeThreads, sv.smem, sv.kstream>>>(q);
    cudaEventRecord(sv.kernel_done, sv.kstream);
    sv.kernel_running = true;
  }
  if (sv.active.empty() && sv.pending.empty())
    __atomic_store_n(&sv.ctl->park, 1u, __ATOMIC_RELEASE);
  return busy || !sv.active.empty();
}

// Uploader thread: scan table, tile bounds, points, a zeroed scratch and the
// ordering's initial box of each admitted request on the copy stream, then
// the request's event. Only copies go to that stream: a memset or a kernel
// there would wait for an SM, and the serving kernel may hold all of them.
void upload_loop(Server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> ul(sv->upmu);
      sv->upcv.wait(ul, [&] { return sv->stop.load() || !sv->upq.empty(); });
      if (sv->upq.empty()) return;  // stopping
      r = sv->upq.front();
      sv->upq.pop_front();
    }
    std::vector<ScanPoint> hs;
    nlos::scan_points_host(r->params, r->g, hs);
    std::vector<TileBound> ht;
    nlos::tile_bounds_host(hs.data(), r->g.S, ht);
    SceneScratch zero{};
    // min words all ones, max words zero (order-preserving bits)
    static const uint32_t box0[kOrderBoxWords] = {~0u, ~0u, ~0u, 0u, 0u, 0u, 0u, 0u};
    cudaError_t e = cudaMemcpyAsync(r->scan, hs.data(), sizeof(ScanPoint) * r->g.S,
                                    cudaMemcpyHostToDevice, sv->cstream);
    if (e == cudaSuccess && !ht.empty())
      e = cudaMemcpyAsync(r->tiles, ht.data(), sizeof(TileBound) * ht.size(),
                          cudaMemcpyHostToDevice, sv->cstream);
    if (e == cudaSuccess && r->g.P)
      e = cudaMemcpyAsync(r->raw, r->pts.data(), sizeof(float) * 8 * r->g.P,
                          cudaMemcpyHostToDevice, sv->cstream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->cells + kOrderCells, box0, sizeof(box0), cudaMemcpyHostToDevice,
                          sv->cstream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->scratch, &zero, sizeof(zero), cudaMemcpyHostToDevice, sv->cstream);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, sv->cstream);
    if (e != cudaSuccess) r->upload_msg = cudaGetErrorString(e);
    r->upload.store(e == cudaSuccess ? 1 : 2, std::memory_order_release);
    sv->cv_work.notify_one();
  }
}

void run(Server* sv) {
  cudaSetDevice(sv->device);
#ifdef __linux__
  // the default timer slack (50 us) would stretch the short sleeps between
  // scheduler passes, and with them every phase transition of a request
  prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->stop.load()) {
    const bool busy = step(*sv);
    if (busy) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(5));
      lk.lock();
    } else {
      sv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
}

}  // namespace serve
}  // namespace nlos

struct nlos_server {
  nlos::serve::Server sv;
};

using namespace nlos;
using namespace nlos::serve;

extern "C" {

nlos_status nlos_server_create(uint64_t hbm_budget_bytes, nlos_server** out) {
  clear_error();
  if (!out) return set_error(NLOS_EINVAL, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes == 0) return set_error(NLOS_EINVAL, "hbm_budget_bytes must be > 0");
  nlos_server* s = new (std::nothrow) nlos_server();
  if (!s) return set_error(NLOS_ENOMEM, "host allocation failed");
  Server& sv = s->sv;
  sv.budget = hbm_budget_bytes;
  auto fail = [&](cudaError_t e, const char* what) {
    if (sv.ctl) cudaFreeHost(sv.ctl);
    if (sv.ring) cudaFreeHost(sv.ring);
    if (sv.jobs) cudaFreeHost(sv.jobs);
    if (sv.status) cudaFreeHost(sv.status);
    if (sv.h_scratch) cudaFreeHost(sv.h_scratch);
    if (sv.d_head) cudaFree(sv.d_head);
    delete s;
    return cuda_error(e, what);
  };
  cudaError_t e = cudaGetDevice(&sv.device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sv.num_sms, cudaDevAttrMultiProcessorCount, sv.device);
  if (e != cudaSuccess) return fail(e, "cudaGetDevice");
  const unsigned flags = cudaHostAllocMapped | cudaHostAllocPortable;
  if ((e = cudaHostAlloc(&sv.ctl, sizeof(Control), flags)) != cudaSuccess) return fail(e, "cudaHostAlloc");
  if ((e = cudaHostAlloc(&sv.ring, sizeof(WorkItem) * 2 * kRing, flags)) != cudaSuccess) return fail(e, "cudaHostAlloc");
  if ((e = cudaHostAlloc(&sv.jobs, sizeof(JobDesc) * kMaxJobs, flags)) != cudaSuccess) return fail(e, "cudaHostAlloc");
  if ((e = cudaHostAlloc(&sv.status, sizeof(JobStatus) * kMaxJobs, flags)) != cudaSuccess) return fail(e, "cudaHostAlloc");
  if ((e = cudaHostAlloc(&sv.h_scratch, sizeof(SceneScratch) * kMaxJobs, cudaHostAllocPortable)) != cudaSuccess)
    return fail(e, "cudaHostAlloc");
  std::memset(sv.ctl, 0, sizeof(Control));
  std::memset(sv.ring, 0xff, sizeof(WorkItem) * 2 * kRing);  // seq = ~0: unpublished
  std::memset(sv.jobs, 0, sizeof(JobDesc) * kMaxJobs);
  std::memset(sv.status, 0, sizeof(JobStatus) * kMaxJobs);
  if ((e = cudaMalloc(&sv.d_head, 2 * sizeof(unsigned long long))) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&sv.dev_args.ctl), sv.ctl, 0)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&sv.dev_args.ring), sv.ring, 0)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&sv.dev_args.jobs), sv.jobs, 0)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&sv.dev_args.status), sv.status, 0)) != cudaSuccess)
    return fail(e, "cudaHostGetDevicePointer");
  sv.dev_args.head = sv.d_head;
  if ((e = cudaMemset(sv.d_head, 0, 2 * sizeof(unsigned long long))) != cudaSuccess) return fail(e, "cudaMemset");
  if ((e = cudaStreamCreateWithFlags(&sv.kstream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "cudaStreamCreate");
  if ((e = cudaStreamCreateWithFlags(&sv.cstream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "cudaStreamCreate");
  if ((e = cudaEventCreateWithFlags(&sv.kernel_done, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "cudaEventCreate");
  sv.smem = (size_t)kCapBw * kTile * 4 + kServeStages * (size_t)kServePpb * sizeof(PointPair) +
            24 * kServeStages + 8 + sizeof(JobDesc) + 64;
  if ((e = cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sv.smem)) != cudaSuccess)
    return fail(e, "cudaFuncSetAttribute");
  cudaDeviceSynchronize();
  for (int i = kMaxJobs - 1; i >= 0; --i) sv.free_slots.push_back(i);
  sv.window[0] = std::min<uint64_t>(kWindowPerSm * (uint64_t)sv.num_sms, kRing / 4);
  sv.window[1] = std::min<uint64_t>(kXWindowPerSm * (uint64_t)sv.num_sms, kRing / 4);
  if (const char* tp = std::getenv("NLOS_SERVE_TRACE")) sv.trace = std::fopen(tp, "a");
  sv.th = std::thread(run, &sv);
  // several uploaders: a copy from pageable memory returns once the data is
  // staged, and requests are independent
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  for (unsigned i = 0; i < std::min(4u, std::max(1u, hw / 4)); ++i)
    sv.uploaders.emplace_back(upload_loop, &sv);
  *out = s;
  return NLOS_OK;
}

nlos_status nlos_serve_submit(nlos_server* server, const nlos_params* params,
                              const float* points_aos8, uint64_t num_points, uint64_t* ticket_out) {
  clear_error();
  if (!server || !params || !ticket_out) return set_error(NLOS_EINVAL, "server, params and ticket_out must not be NULL");
  if (num_points && !points_aos8) return set_error(NLOS_EINVAL, "points_aos8 is NULL");
  Request* r = new (std::nothrow) Request();
  if (!r) return set_error(NLOS_ENOMEM, "host allocation failed");
  nlos_status st = resolve_params(*params, num_points, r->g);
  if (st != NLOS_OK) {
    delete r;
    return st;
  }
  r->params = *params;
  if (r->g.bin_mode == NLOS_BIN_NEAREST && jitter_radius(r->g.sigma) > 64) {
    delete r;
    return set_error(NLOS_EINVAL, "jitter too wide");
  }
  try {
    r->pts.assign(points_aos8, points_aos8 + 8 * num_points);
  } catch (...) {
    delete r;
    return set_error(NLOS_ENOMEM, "host allocation failed");
  }
  if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) {
    delete r;
    return set_error(NLOS_ECUDA, "event creation failed");
  }
  Server& sv = server->sv;
  {
    std::lock_guard<std::mutex> lk(sv.mu);
    r->ticket = sv.next_ticket++;
    r->t_submit = Clock::now();
    sv.reqs[r->ticket] = r;
    sv.pending.push_back(r);
  }
  sv.cv_work.notify_one();
  *ticket_out = r->ticket;
  return NLOS_OK;
}

nlos_status nlos_serve_poll(nlos_server* server, uint64_t ticket, int wait_ms,
                            const float** tau_dev_out, const uint32_t** counts_dev_out,
                            nlos_stats* stats) {
  clear_error();
  if (!server) return set_error(NLOS_EINVAL, "server is NULL");
  if (stats && stats->struct_size != sizeof(nlos_stats))
    return set_error(NLOS_EINVAL, "nlos_stats.struct_size does not match this library");
  Server& sv = server->sv;
  std::unique_lock<std::mutex> lk(sv.mu);
  auto it = sv.reqs.find(ticket);
  if (it == sv.reqs.end()) return set_error(NLOS_ENOTFOUND, "unknown ticket");
  Request* r = it->second;
  auto finished = [&] { return r->state == R_DONE || r->state == R_FAILED || r->state == R_CANCELLED; };
  if (!finished() && wait_ms > 0)
    sv.cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), finished);
  if (!finished()) return set_error(NLOS_EBUSY, "pending");
  if (r->state == R_CANCELLED) return set_error(NLOS_ECANCELLED, "cancelled");
  if (r->state == R_FAILED) return set_error(r->status, r->msg);
  if (tau_dev_out) *tau_dev_out = r->tau;
  if (counts_dev_out) *counts_dev_out = r->counts;
  if (stats) *stats = r->stats;
  return NLOS_OK;
}

nlos_status nlos_serve_release(nlos_server* server, uint64_t ticket) {
  clear_error();
  if (!server) return set_error(NLOS_EINVAL, "server is NULL");
  Server& sv = server->sv;
  std::lock_guard<std::mutex> lk(sv.mu);
  auto it = sv.reqs.find(ticket);
  if (it == sv.reqs.end()) return set_error(NLOS_ENOTFOUND, "unknown ticket");
  Request* r = it->second;
  if (r->state == R_PENDING) {
    sv.pending.erase(std::find(sv.pending.begin(), sv.pending.end(), r));
    destroy_request(sv, r);
  } else if (r->state == R_DONE || r->state == R_FAILED || r->state == R_CANCELLED) {
    destroy_request(sv, r);
  } else {
    // admitted: the ticket is gone now; the memory is freed once the work
    // already published for it has completed on the device
    r->release_on_done = true;
    sv.reqs.erase(it);
  }
  return NLOS_OK;
}

nlos_status nlos_server_destroy(nlos_server* server) {
  clear_error();
  if (!server) return set_error(NLOS_EINVAL, "server is NULL");
  Server& sv = server->sv;
  {
    // let admitted work finish (bounded), then park the kernel
    auto t0 = Clock::now();
    std::unique_lock<std::mutex> lk(sv.mu);
    while (!sv.active.empty() && Clock::now() - t0 < std::chrono::seconds(30)) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::milliseconds(1));
      lk.lock();
    }
    for (Request* r : sv.pending) r->state = R_CANCELLED;
    sv.pending.clear();
    __atomic_store_n(&sv.ctl->park, 1u, __ATOMIC_RELEASE);
  }
  sv.stop.store(true);
  sv.cv_work.notify_all();
  if (sv.th.joinable()) sv.th.join();
  {
    std::lock_guard<std::mutex> ul(sv.upmu);
    sv.upcv.notify_all();
  }
  for (std::thread& t : sv.uploaders)
    if (t.joinable()) t.join();
  cudaStreamSynchronize(sv.kstream);  // the kernel exits once parked (bounded waits)
  cudaStreamSynchronize(sv.cstream);
  std::vector<Request*> all;
  for (auto& kv : sv.reqs) all.push_back(kv.second);
  for (Request* r : all) destroy_request(sv, r);
  cudaStreamSynchronize(sv.cstream);
  cudaEventDestroy(sv.kernel_done);
  cudaStreamDestroy(sv.kstream);
  cudaStreamDestroy(sv.cstream);
  cudaFree(sv.d_head);
  cudaFreeHost(sv.ctl);
  cudaFreeHost(sv.ring);
  cudaFreeHost(sv.jobs);
  cudaFreeHost(sv.status);
  cudaFreeHost(sv.h_scratch);
  if (sv.trace) std::fclose(sv.trace);
  delete server;
  return NLOS_OK;
}

nlos_status nlos_server_inject(nlos_server* server, int fault) {
  clear_error();
  if (!server) return set_error(NLOS_EINVAL, "server is NULL");
  if (fault < 0 || fault > 2) return set_error(NLOS_EINVAL, "unknown fault");
  std::lock_guard<std::mutex> lk(server->sv.mu);
  server->sv.inject = fault;
  return NLOS_OK;
}

nlos_status nlos_server_stats(nlos_server* server, uint64_t* resident_bytes, uint32_t* pending,
                              uint32_t* active) {
  clear_error();
  if (!server) return set_error(NLOS_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(server->sv.mu);
  if (resident_bytes) *resident_bytes = server->sv.resident;
  if (pending) *pending = (uint32_t)server->sv.pending.size();
  if (active) *active = (uint32_t)server->sv.active.size();
  return NLOS_OK;
}

nlos_status nlos_server_device_cycles(nlos_server* server, uint64_t cycles_out[3]) {
  clear_error();
  if (!server || !cycles_out) return set_error(NLOS_EINVAL, "server or cycles_out is NULL");
  const Control* c = server->sv.ctl;
  for (int k = 0; k < 3; ++k) cycles_out[k] = __atomic_load_n(&c->cycles[k], __ATOMIC_ACQUIRE);
  return NLOS_OK;
}

}  // extern "C"
