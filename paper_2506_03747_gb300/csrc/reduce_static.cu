// nlos_reduce_static: the cube reduction of nlos_reduce without any device
// allocation, for callers that cannot allocate device memory at the point of
// the call (their device memory is already reserved up front by another
// allocator, such as a framework's caching pool, so a fresh cudaMalloc can
// fail even while memory sits unused in that pool; or they run a
// latency-bound loop in which the device-wide synchronisation that
// cudaMalloc/cudaFree can cause is not acceptable).
//
// Instead of a scratch buffer allocated per call, the per-transient partial
// results live in a fixed array in this library's device image. Every device
// that loads the library holds that array (kStaticMaxTraces x 24 bytes,
// 1.5 MiB) until the process exits.
//
// Two kernels, both deterministic (no atomics):
//  1. one warp per transient: FP64 energy (written to energy_dev if given)
//     and the transient's max, FP64 sum and sum of squares into the array;
//  2. one CTA combines the partials of transients [0, num_traces) in a fixed
//     order and writes {max, sum, sum of squares} to stats_dev.
// Pass 1 overwrites every partial that pass 2 reads, so nothing needs to be
// cleared between calls; calls whose kernels overlap on the GPU (different
// streams, no ordering) race on the array.
#include "common.cuh"
#include "reduce_core.cuh"

#include <mutex>

namespace nlos {
namespace {

constexpr uint64_t kStaticMaxTraces = 65536;

struct __align__(8) TracePartial {
  double sum;
  double sumsq;
  float max;
  float pad;
};
static_assert(sizeof(TracePartial) == 24, "partial layout");

static __device__ __align__(256) TracePartial g_partials[kStaticMaxTraces];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
TracePartial* g_dev_ptr[kMaxDevices] = {};
void* g_dev_ctx[kMaxDevices] = {};  // the context each address was looked up in

// The calling thread's current CUDA context (the driver's cuCtxGetCurrent,
// found through the runtime so that the library needs no link to the driver
// library), or null if none is current or the call is unavailable.
void* current_context() {
  using CtxGetCurrent = int (*)(void**);
  static CtxGetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return static_cast<CtxGetCurrent>(nullptr);
    return reinterpret_cast<CtxGetCurrent>(f);
  }();
  void* ctx = nullptr;
  if (fn && fn(&ctx) != 0) ctx = nullptr;
  return ctx;
}

// Device address of g_partials on the current device, looked up once per
// device and context (host code must not use the symbol itself as an
// address). A context destroyed and made anew (cudaDeviceReset) loads the
// module again, so an address is reused only in the context it came from.
cudaError_t partials_address(TracePartial** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  void* ctx = current_context();
  if (!g_dev_ptr[dev] || !ctx || ctx != g_dev_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);  // makes the device's context current
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = static_cast<TracePartial*>(p);
    g_dev_ctx[dev] = ctx ? ctx : current_context();
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

__global__ void partials_kernel(const float* __restrict__ tau, uint64_t traces, uint32_t B,
                                double* energy, TracePartial* part) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < traces;
       t += warps) {
    double s, q;
    float m;
    trace_sums(tau + t * B, B, lane, s, q, m);
    if (lane == 0) {
      if (energy) energy[t] = s;
      part[t].sum = s;
      part[t].sumsq = q;
      part[t].max = m;
    }
  }
}

// One CTA of 1024 threads: thread i folds partials i, i + 1024, ... in order,
// then a fixed shared-memory tree combines the 1024 results.
__global__ void __launch_bounds__(1024) combine_kernel(const TracePartial* part, uint64_t traces,
                                                       double* stats) {
  __shared__ double ss[1024];
  __shared__ double sq[1024];
  __shared__ float sm[1024];
  double s = 0.0, q = 0.0;
  float m = 0.0f;
  for (uint64_t t = threadIdx.x; t < traces; t += blockDim.x) {
    s += part[t].sum;
    q += part[t].sumsq;
    m = fmaxf(m, part[t].max);
  }
  ss[threadIdx.x] = s;
  sq[threadIdx.x] = q;
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      ss[threadIdx.x] += ss[threadIdx.x + w];
      sq[threadIdx.x] += sq[threadIdx.x + w];
      sm[threadIdx.x] = fmaxf(sm[threadIdx.x], sm[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[0] = (double)sm[0];
    stats[1] = ss[0];
    stats[2] = sq[0];
  }
}

}  // namespace
}  // namespace nlos

using namespace nlos;

extern "C" nlos_status nlos_reduce_static(const float* tau_dev, uint64_t num_traces,
                                          uint32_t num_bins, double* energy_dev,
                                          double* stats_dev, void* cuda_stream) {
  clear_error();
  if (!tau_dev && num_traces) return set_error(NLOS_EINVAL, "tau_dev is NULL");
  if (num_traces > kStaticMaxTraces)
    return set_error(NLOS_EINVAL,
                     "num_traces exceeds the static scratch of nlos_reduce_static (at most 65536 "
                     "transients per call); use nlos_reduce");
  if (num_bins == 0 && num_traces) return set_error(NLOS_EINVAL, "num_bins must be > 0");
  if ((num_bins & 3u) == 0u && (reinterpret_cast<uintptr_t>(tau_dev) & 15u))
    return set_error(NLOS_EINVAL, "tau_dev must be 16-byte aligned");
  TracePartial* part = nullptr;
  NLOS_CUDA_TRY(partials_address(&part));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (num_traces) {
    int dev = 0, sms = 0;
    NLOS_CUDA_TRY(cudaGetDevice(&dev));
    NLOS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t want = (num_traces + 7) / 8;
    const unsigned blocks = (unsigned)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
    partials_kernel<<<blocks, 256, 0, st>>>(tau_dev, num_traces, num_bins, energy_dev, part);
    NLOS_CUDA_TRY(cudaGetLastError());
  }
  if (stats_dev) {
    combine_kernel<<<1, 1024, 0, st>>>(part, num_traces, stats_dev);
    NLOS_CUDA_TRY(cudaGetLastError());
  }
  return NLOS_OK;
}
