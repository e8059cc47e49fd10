// Detector model kernels of the GB300 NLOS simulator (arXiv 2506.03747):
//  * Gaussian timing jitter per transient (Eq. 16/17, Algorithm 1 step 2.3);
//  * per-transient FP64 energy, and the cube's maximum / FP64 sum and sum of
//    squares that set the noise scale;
//  * seeded Poisson photon + dark-count noise (Eq. 18/19, Algorithm 1 step 2.4)
//    from per-bin Philox4x32-10 counter streams.
// All three are HBM-streaming kernels: coalesced row-wise reads and writes,
// grids sized to the SM count.
#include "common.cuh"
#include "device_util.cuh"
#include "noise_core.cuh"
#include "reduce_core.cuh"

#include <cmath>

namespace nlos {

// ---------------------------------------------------------------------------
// Jitter taps: sigma in bins, R = ceil(2 sigma), k = 2R + 1 (Eq. 17), sampled
// Gaussian exp(-j^2 / (2 sigma^2)) normalised to sum 1 (computed in FP64 on
// the host, stored FP32). sigma = 0 gives the identity (k = 1).
// ---------------------------------------------------------------------------
int jitter_taps(double sigma, float* taps, int max_taps) {
  const int R = jitter_radius(sigma);
  const int k = 2 * R + 1;
  if (k > max_taps) return -k;
  if (R == 0) {
    taps[0] = 1.0f;
    return 1;
  }
  static thread_local double t[4097];
  double sum = 0.0;
  for (int j = -R; j <= R; ++j) {
    t[j + R] = std::exp(-(double)j * (double)j / (2.0 * sigma * sigma));
    sum += t[j + R];
  }
  for (int j = 0; j < k; ++j) taps[j] = (float)(t[j] / sum);
  return k;
}

void jitter_tails(const float* taps, int R, float* tail) {
  double acc = 0.0;  // running sum from the outermost tap inwards
  for (int k = R - 1; k >= 0; --k) {
    acc += (double)taps[R + k + 1];
    tail[k] = (float)acc;
  }
}

constexpr int kJitterMaxTaps = 2049;  // R <= 1024 bins
constexpr int kJitterTile = 1024;

struct JitterArgs {
  const float* in;
  float* out;
  uint64_t traces;
  uint32_t B;
  int R;
  int replicate;  // 1: the edge bins continue outside the trace
  float taps[kJitterMaxTaps];
};

// One CTA = one run of kJitterTile output bins of one trace; the input run
// with its R-bin halo is staged in shared memory (zero outside the trace).
__global__ void jitter_kernel(const __grid_constant__ JitterArgs a) {
  extern __shared__ float sm[];  // [kJitterTile + 2R] input
  const uint32_t tiles_per_trace = (a.B + kJitterTile - 1) / kJitterTile;
  const uint64_t t = blockIdx.x / tiles_per_trace;
  const int b0 = (int)(blockIdx.x % tiles_per_trace) * kJitterTile;
  const float* row = a.in + t * a.B;
  for (int i = threadIdx.x; i < kJitterTile + 2 * a.R; i += blockDim.x) {
    const int b = b0 - a.R + i;
    if (a.replicate) sm[i] = row[min(max(b, 0), (int)a.B - 1)];
    else sm[i] = (b >= 0 && b < (int)a.B) ? row[b] : 0.0f;
  }
  __syncthreads();
  float* orow = a.out + t * a.B;
  for (int i = threadIdx.x; i < kJitterTile; i += blockDim.x) {
    const int b = b0 + i;
    if (b >= (int)a.B) break;
    float acc = 0.0f;
    // out[b] = sum_j taps[j + R] * in[b - j]; in[b - j] sits at sm[i + R - j]
    for (int j = -a.R; j <= a.R; ++j) acc = fmaf(a.taps[j + a.R], sm[i + a.R - j], acc);
    orow[b] = acc;
  }
}

cudaError_t launch_jitter(const float* in, float* out, uint64_t traces, uint32_t B, double sigma,
                          int replicate, cudaStream_t st) {
  if (traces == 0 || B == 0) return cudaSuccess;
  JitterArgs a;
  a.in = in;
  a.out = out;
  a.traces = traces;
  a.B = B;
  a.replicate = replicate;
  const int k = jitter_taps(sigma, a.taps, kJitterMaxTaps);
  if (k < 0) return cudaErrorInvalidValue;
  a.R = (k - 1) / 2;
  const uint64_t blocks = traces * ((B + kJitterTile - 1) / kJitterTile);
  const size_t smem = sizeof(float) * (kJitterTile + 2 * a.R);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(jitter_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  jitter_kernel<<<(unsigned)blocks, 256, smem, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reductions: one warp per transient. energy[t] = sum_b tau[t][b] to FP64
// accuracy (trace_sums, reduce_core.cuh: error-free FP32 pair sums per lane);
// the cube's maximum, FP64 sum and sum of squares are combined per CTA in
// shared memory, then one atomicMax on the float bits (tau >= 0 orders like
// its bits) and two double atomicAdds per CTA (per-warp atomics on the same
// three words serialised in L2).
// ---------------------------------------------------------------------------
constexpr int kReduceThreads = 256;

__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(const float* __restrict__ tau,
                                                                uint64_t traces, uint32_t B,
                                                                double* energy,
                                                                SceneScratch* scratch) {
  __shared__ double s_sum[kReduceThreads / 32], s_sq[kReduceThreads / 32];
  __shared__ float s_max[kReduceThreads / 32];
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  double csum = 0.0, csq = 0.0;
  float cmax = 0.0f;
  for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < traces;
       t += warps) {
    double s, q;
    float m;
    trace_sums(tau + t * B, B, lane, s, q, m);
    if (lane == 0 && energy) energy[t] = s;
    csum += s;
    csq += q;
    cmax = fmaxf(cmax, m);
  }
  if (!scratch) return;
  const int warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_sum[warp] = csum;
    s_sq[warp] = csq;
    s_max[warp] = cmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      csum += s_sum[w];
      csq += s_sq[w];
      cmax = fmaxf(cmax, s_max[w]);
    }
    atomicMax(&scratch->peak_bits, __float_as_uint(cmax));
    atomicAdd(&scratch->sum, csum);
    atomicAdd(&scratch->sumsq, csq);
  }
}

__global__ void stats_out_kernel(const SceneScratch* scratch, double* stats) {
  stats[0] = (double)__uint_as_float(scratch->peak_bits);
  stats[1] = scratch->sum;
  stats[2] = scratch->sumsq;
}

cudaError_t launch_stats_out(const SceneScratch* scratch, double* stats, cudaStream_t st) {
  stats_out_kernel<<<1, 1, 0, st>>>(scratch, stats);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const float* tau, uint64_t traces, uint32_t B, double* energy,
                          SceneScratch* scratch, cudaStream_t st) {
  if (traces == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t want = (traces + 7) / 8;
  const unsigned blocks = (unsigned)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
  reduce_kernel<<<blocks, kReduceThreads, 0, st>>>(tau, traces, B, energy, scratch);
  return cudaGetLastError();
}

struct NoiseArgs {
  const float* tau;
  uint32_t* counts;
  uint64_t n;
  uint64_t index_base;
  uint64_t seed;
  uint32_t tag;
  float scale, dark;          // used when scratch == nullptr
  SceneScratch* scratch;      // else: scale from the reduced cube
  int mode;                   // nlos_noise_mode (scratch path)
  float peak_photons, dark_cfg, nr_db;
  const double* cube_stats;   // part of a larger cube: {max, sum, sumsq} of the whole
  uint64_t cube_bins;         // bins of the whole cube
  DeferList defer;            // deferred bright bins (defer.hdr null: one pass)
};

// CTAs of 7 warps, kNoiseBlocksPerSm resident per SM (32 registers), up to
// NLOS_NOISE_WAVES waves of them. A thread samples one group of four bins at a
// time (one Philox block for the four first draws, a 16-byte load and store);
// warp w takes the 32 consecutive groups of chunk c = w, w + W, w + 2W, ...
// (lane = group, coalesced). The warp count W is odd, so the stride W * 128
// bins moves a warp's bins through the time indices of the transients: a
// bin's cost grows with its lambda and the bright bins sit at a few time
// indices, and a stride that is a multiple of the bin count (a wave of
// 256-thread blocks of 1024-bin transients: 1216 * 256 = 304 * 1024) gave some
// warps every bright bin of the cube (ncu: SMs 40% active, ALU pipe from 19%
// to 99% over the SMs). With up to 16 waves a thread mostly takes one group,
// and the CTAs that meet bright bins are the ones that run long (heightfield128
// 0.139 ms against 0.156 ms with one wave and a longer stride loop; union64
// 0.060 against 0.057). No atomics and no divisions in the loop; 1/k of the
// inversion search from a shared table.
constexpr int kNoiseWarps = 7;
constexpr int kNoiseThreads = 32 * kNoiseWarps;
constexpr int kNoiseBlocksPerSm = 8;
#ifndef NLOS_NOISE_WAVES
#define NLOS_NOISE_WAVES 16  // resident waves of CTAs at most (the rest by the grid stride)
#endif

#ifndef NLOS_NOISE_DEFER
#define NLOS_NOISE_DEFER 1  // bins with lambda >= 30 sampled by a second kernel
#endif

// The noise scale and dark level of a launch (the same in every thread and
// in both kernels of a launch).
__device__ __forceinline__ void launch_scale(const NoiseArgs& a, float& scale, float& dark) {
  scale = a.scale;
  dark = a.dark;
  if (a.cube_stats) {
    scale = noise_scale_of((float)a.cube_stats[0], a.cube_stats[1], a.cube_stats[2], a.mode,
                           a.peak_photons, a.nr_db, a.cube_bins);
    dark = a.dark_cfg;
  } else if (a.scratch) {
    scale = noise_scale_from(a.scratch, a.mode, a.peak_photons, a.nr_db, a.n);
    dark = a.dark_cfg;
  }
}

template <bool DEFER>
__global__ void __launch_bounds__(kNoiseThreads, kNoiseBlocksPerSm) noise_kernel(const NoiseArgs a) {
  // one table per warp, so that no CTA barrier is needed (CTAs are short)
  __shared__ float rcp_tab[kNoiseWarps][kRcpTable];
  float* rcp = rcp_tab[threadIdx.x >> 5];
  fill_rcp_table(rcp, threadIdx.x & 31, 32);
  __syncwarp();
  float scale, dark;
  launch_scale(a, scale, dark);
  if (a.scratch && blockIdx.x == 0 && threadIdx.x == 0) {
    a.scratch->scale = scale;
    a.scratch->dark = dark;
  }
  const uint64_t stride = (uint64_t)gridDim.x * kNoiseWarps * 32;
  const uint64_t j0 = ((uint64_t)blockIdx.x * kNoiseWarps + (threadIdx.x >> 5)) * 32 +
                      (threadIdx.x & 31);
  noise_groups<DEFER>(a.tau, a.counts, 0, a.n, a.index_base, scale, dark, a.seed, a.tag, rcp, j0,
                      stride, &a.defer);
}

// Second pass (after noise_kernel, in stream order): one thread per listed
// bin (the cube's bright bins, about 1% of them), then one warp per listed
// region of a warp whose bins did not fit the list.
constexpr int kDeferThreads = 256;

__global__ void __launch_bounds__(kDeferThreads) noise_deferred_kernel(const NoiseArgs a) {
  __shared__ float rcp_tab[kDeferThreads / 32][kRcpTable];  // one table per warp
  float* rcp = rcp_tab[threadIdx.x >> 5];
  fill_rcp_table(rcp, threadIdx.x & 31, 32);
  __syncwarp();
  float scale, dark;
  launch_scale(a, scale, dark);
  const DeferList& d = a.defer;
  const unsigned long long claimed = *(volatile unsigned long long*)&d.hdr[0];
  const unsigned long long nd = claimed < d.cap ? claimed : d.cap;
  const uint64_t nt = (uint64_t)gridDim.x * kDeferThreads;
  for (uint64_t k = (uint64_t)blockIdx.x * kDeferThreads + threadIdx.x; k < nd; k += nt) {
    const uint32_t l = d.bins[k];
    if (l != kDeferredCount)
      noise_deferred_bin(a.tau, a.counts, l, a.index_base, scale, dark, a.seed, a.tag, rcp);
  }
  const unsigned long long nr = *(volatile unsigned long long*)&d.hdr[1];
  const uint64_t nw = nt / 32;
  for (uint64_t k = (uint64_t)blockIdx.x * (kDeferThreads / 32) + (threadIdx.x >> 5); k < nr;
       k += nw)
    noise_deferred_warp(a.tau, a.counts, a.n, d.regions[k], a.index_base, scale, dark, a.seed,
                        a.tag, rcp);
}

cudaError_t launch_noise_impl(const NoiseArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t groups = ((a.index_base + a.n + 3) >> 2) - (a.index_base >> 2);
  const uint64_t want = (groups + kNoiseThreads - 1) / kNoiseThreads;
  const uint64_t wave = (uint64_t)sms * kNoiseBlocksPerSm * NLOS_NOISE_WAVES;
  uint64_t blocks = want < wave ? want : wave;
  if (blocks > 1 && (blocks & 1u) == 0) --blocks;  // an odd number of warps (7 per block)
  // the deferred-bin lists: the header, a dense list of local indices for
  // about 3% of the bins, and one entry per warp region for the warps whose
  // bins overflow it (the regions of 32 groups cover the launch's groups, plus
  // one for an unaligned start); one stream-ordered allocation, freed after
  // the second pass. Without it (or for parts of 2^32 - 1 bins or more) every
  // bin is sampled in one pass.
  NoiseArgs b = a;
  b.defer = DeferList{};
  cudaError_t e = cudaSuccess;
  if (NLOS_NOISE_DEFER && a.n < 0xFFFFFFFFull) {
    const uint64_t cap = std::min<uint64_t>(a.n, a.n / 32 + 4096);
    const uint64_t n_reg = groups / 32 + 2;
    const size_t bytes = 2 * sizeof(unsigned long long) + n_reg * sizeof(unsigned long long) +
                         ((cap * sizeof(uint32_t) + 15) & ~(size_t)15);
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, bytes, st) != cudaSuccess) {
      (void)cudaGetLastError();  // no lists: one pass
    } else if ((e = cudaMemsetAsync(buf, 0, 2 * sizeof(unsigned long long), st)) !=
               cudaSuccess) {
      cudaFreeAsync(buf, st);
      return e;
    } else {
      b.defer.hdr = static_cast<unsigned long long*>(buf);
      b.defer.regions = b.defer.hdr + 2;
      b.defer.bins = reinterpret_cast<uint32_t*>(b.defer.regions + n_reg);
      b.defer.cap = (uint32_t)cap;
    }
  }
  if (b.defer.hdr)
    noise_kernel<true><<<(unsigned)blocks, kNoiseThreads, 0, st>>>(b);
  else
    noise_kernel<false><<<(unsigned)blocks, kNoiseThreads, 0, st>>>(b);
  e = cudaGetLastError();
  if (b.defer.hdr) {
    if (e == cudaSuccess) {
      noise_deferred_kernel<<<(unsigned)(sms * 4), kDeferThreads, 0, st>>>(b);
      e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(b.defer.hdr, st);
    if (e == cudaSuccess) e = ef;
  }
  return e;
}

cudaError_t launch_noise(const float* tau, uint64_t n, float scale, float dark, uint64_t seed,
                         uint32_t tag, uint64_t index_base, uint32_t* counts, cudaStream_t st) {
  NoiseArgs a{};
  a.tau = tau;
  a.counts = counts;
  a.n = n;
  a.index_base = index_base;
  a.seed = seed;
  a.tag = tag;
  a.scale = scale;
  a.dark = dark;
  a.scratch = nullptr;
  return launch_noise_impl(a, st);
}

cudaError_t launch_noise_scene(const float* tau, uint64_t n, SceneScratch* scratch, int mode,
                               float peak_photons, float dark, float nr_db, uint64_t seed,
                               uint32_t tag, uint32_t* counts, cudaStream_t st,
                               uint64_t index_base, const double* cube_stats,
                               uint64_t cube_bins) {
  NoiseArgs a{};
  a.tau = tau;
  a.counts = counts;
  a.n = n;
  a.index_base = index_base;
  a.cube_stats = cube_stats;
  a.cube_bins = cube_bins;
  a.seed = seed;
  a.tag = tag;
  a.scratch = scratch;
  a.mode = mode;
  a.peak_photons = peak_photons;
  a.dark_cfg = dark;
  a.nr_db = nr_db;
  return launch_noise_impl(a, st);
}

// ---------------------------------------------------------------------------
// Raw Philox words (parity testing of the device generator).
// ---------------------------------------------------------------------------
__global__ void philox_kernel(const uint4* ctr, uint64_t n, uint32_t k0, uint32_t k1, uint4* out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = philox4x32_10(ctr[i], k0, k1);
}

cudaError_t launch_philox(const uint32_t* ctr, uint64_t n, uint32_t k0, uint32_t k1,
                          uint32_t* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const uint64_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)(want < 4096 ? want : 4096);
  philox_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const uint4*>(ctr), n, k0, k1,
                                        reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

}  // namespace nlos
