// Throughput microbenchmarks of the GB300 units the forward pair sum is bound
// by (its roofline denominators): FP32 FMA (scalar and packed FP32x2), the
// MUFU square root / reciprocal / reciprocal square root estimates, shared
// memory loads, and shared-memory reductions in the layout the forward's
// histograms use ([row][32] words: lane l always hits bank l, rows differ per
// lane). Each kernel runs one 1024-thread CTA per SM; thread 0 of every CTA
// reads clock64 around the timed loop (between two CTA barriers), so the
// results are element operations per SM clock per SM, independent of the
// clock the GPU happens to run at.
#include "common.cuh"
#include "device_util.cuh"

#include <vector>

namespace nlos {
namespace {

enum PeakKind {
  PK_FFMA = 0,     // fmaf, 8 independent chains per thread
  PK_FFMA2,        // __ffma2_rn (two FMAs per lane and instruction)
  PK_SQRT,         // sqrt.approx.ftz.f32
  PK_RCP,          // rcp.approx.ftz.f32 (with one FP32 add a step)
  PK_RSQRT,        // rsqrt.approx.ftz.f32
  PK_LDS128,       // ld.shared.v4.f32, every lane the same address (broadcast)
  PK_RED_F32,      // red.shared.add.f32, all lanes
  PK_RED_U32,      // red.shared.add.u32, all lanes
  PK_RED_U64,      // red.shared.add.u64, all lanes ([row][32] 8-byte words)
  PK_RMW_F32,      // ld.shared + add + st.shared (no atomicity), all lanes
  PK_RED_F32_Q,    // red.shared.add.f32, one lane in four
  PK_RED_U32_Q,    // red.shared.add.u32, one lane in four
  PK_DFMA,         // fma on doubles, 8 independent chains per thread
  PK_ATOM_F32,     // atom.shared.add.f32 (old value returned), all lanes
  PK_COUNT
};

constexpr int kPeakThreads = 1024;
constexpr int kPeakRows = 512;
constexpr int kPeakChains = 8;

__device__ __forceinline__ uint32_t hash_row(uint32_t a) {
  a ^= a >> 16;
  a *= 0x7feb352dU;
  a ^= a >> 15;
  a *= 0x846ca68bU;
  a ^= a >> 16;
  return a % kPeakRows;
}

// volatile: each estimate is issued as written (rcp(rcp(x)) is not folded)
__device__ __forceinline__ float mufu_sqrt(float x) {
  float r;
  asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float mufu_rcp(float x) {
  float r;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float mufu_rsqrt(float x) {
  float r;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int K>
__global__ void __launch_bounds__(kPeakThreads, 1)
    peak_kernel(int iters, float seed, float* sink, long long* cycles) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // rows of this thread's kPeakChains reduction targets (per lane: rows differ
  // across lanes and warps, the bank is always the lane's)
  uint32_t addr[kPeakChains];
  const uint32_t base = smem_addr(smem);
  const uint32_t word = (K == PK_RED_U64) ? 8u : 4u;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k)
    addr[k] = base + hash_row((uint32_t)(warp * 977 + k * 131 + lane * 7 + blockIdx.x)) * 32u * word +
              (uint32_t)lane * word;
  for (int i = tid; i < kPeakRows * 32 * 2; i += blockDim.x) reinterpret_cast<float*>(smem)[i] = 0.f;
  float acc[kPeakChains];
  float2 acc2[kPeakChains];
  double accd[K == PK_DFMA ? kPeakChains : 1];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) {
    acc[k] = seed + 0.001f * (float)(k + 1) + 1e-6f * (float)tid;
    acc2[k] = make_float2(acc[k], acc[k] + 0.5f);
    if (K == PK_DFMA) accd[k] = (double)acc[k];
  }
  const float m = 0.999f, c = 1e-3f;
  __syncthreads();
  long long t0 = 0;
  if (tid == 0) t0 = clock64();
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
    if (K == PK_FFMA) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) acc[k] = fmaf(acc[k], m, c);
    } else if (K == PK_DFMA) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) accd[k] = fma(accd[k], 0.999, 1e-3);
    } else if (K == PK_FFMA2) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k)
        acc2[k] = __ffma2_rn(acc2[k], make_float2(m, m), make_float2(c, c));
    } else if (K == PK_SQRT) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) acc[k] = mufu_sqrt(acc[k]);
    } else if (K == PK_RCP) {
      // 1 / (1 + x): a chain the compiler cannot fold (1 / (1 / x) could be)
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) acc[k] = mufu_rcp(acc[k] + 1.0f);
    } else if (K == PK_RSQRT) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) acc[k] = mufu_rsqrt(acc[k]);
    } else if (K == PK_LDS128) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) {
        float4 v;
        const uint32_t a = base + (uint32_t)(((it * kPeakChains + k) & 1023) * 16);
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "r"(a));
        acc[k] += v.x;  // keeps the loads live (one FADD per load)
      }
    } else if (K == PK_RED_F32 || K == PK_RED_F32_Q) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) {
        const uint32_t on = (K == PK_RED_F32) ? 1u : (((lane + k) & 3) == 0 ? 1u : 0u);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n @p red.shared.add.f32 [%0], %1;\n}\n" ::"r"(
                addr[k]),
            "f"(acc[k]), "r"(on)
            : "memory");
      }
    } else if (K == PK_ATOM_F32) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) {
        float old;
        asm volatile("atom.shared.add.f32 %0, [%1], %2;"
                     : "=f"(old)
                     : "r"(addr[k]), "f"(acc[k])
                     : "memory");
        acc[k] += old * 0.0f;  // keeps the returned value live
      }
    } else if (K == PK_RED_U32 || K == PK_RED_U32_Q) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) {
        const uint32_t on = (K == PK_RED_U32) ? 1u : (((lane + k) & 3) == 0 ? 1u : 0u);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n @p red.shared.add.u32 [%0], %1;\n}\n" ::"r"(
                addr[k]),
            "r"((uint32_t)k + 1u), "r"(on)
            : "memory");
      }
    } else if (K == PK_RED_U64) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k)
        asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(addr[k]), "l"((unsigned long long)k + 1ull)
                     : "memory");
    } else if (K == PK_RMW_F32) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k)
        asm volatile(
            "{\n .reg .f32 t;\n ld.shared.f32 t, [%0];\n add.f32 t, t, %1;\n st.shared.f32 [%0], t;\n}\n" ::"r"(
                addr[k]),
            "f"(acc[k])
            : "memory");
    }
  }
  __syncthreads();
  if (tid == 0) cycles[blockIdx.x] = clock64() - t0;
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += acc[k] + acc2[k].x + acc2[k].y;
  if (K == PK_DFMA)
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += (float)accd[k];
  sink[(size_t)blockIdx.x * blockDim.x + tid] = s;
}

// element operations of one thread per loop iteration
constexpr double ops_per_iter(int k) {
  return k == PK_FFMA2 ? 2.0 * kPeakChains
         : (k == PK_RED_F32_Q || k == PK_RED_U32_Q) ? kPeakChains / 4.0
                                                     : (double)kPeakChains;
}

constexpr int iters_of(int k) {
  return k == PK_DFMA ? 256
         : (k == PK_FFMA || k == PK_FFMA2) ? 8192
         : (k == PK_SQRT || k == PK_RCP || k == PK_RSQRT || k == PK_LDS128) ? 1024
                                                                            : 256;
}

using PeakFn = void (*)(int, float, float*, long long*);

template <int K>
cudaError_t run_one(int n_sm, float* sink, long long* cyc_dev, std::vector<long long>& cyc,
                    cudaStream_t st, double& rate) {
  const size_t smem = (size_t)kPeakRows * 32 * 8;  // enough for the 8-byte rows
  PeakFn fn = peak_kernel<K>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int iters = iters_of(K);
  // one warm-up launch (clocks ramp, instruction cache), one timed
  for (int rep = 0; rep < 2; ++rep) {
    fn<<<n_sm, kPeakThreads, smem, st>>>(rep == 0 ? 4 : iters, 1.0f, sink, cyc_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  e = cudaMemcpyAsync(cyc.data(), cyc_dev, sizeof(long long) * n_sm, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  double sum = 0.0;
  for (int i = 0; i < n_sm; ++i) sum += (double)cyc[i];
  const double mean_cycles = sum / n_sm;
  rate = (double)kPeakThreads * iters * ops_per_iter(K) / mean_cycles;
  return cudaSuccess;
}

}  // namespace
}  // namespace nlos

using namespace nlos;

extern "C" nlos_status nlos_measure_peaks(nlos_peaks* out, void* cuda_stream) {
  clear_error();
  if (!out || out->struct_size < sizeof(nlos_peaks))
    return set_error(NLOS_EINVAL, "nlos_measure_peaks: out is null or struct_size too small");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0, n_sm = 0;
  NLOS_CUDA_TRY(cudaGetDevice(&dev));
  NLOS_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  float* sink = nullptr;
  long long* cyc_dev = nullptr;
  NLOS_CUDA_TRY(cudaMallocAsync(&sink, sizeof(float) * (size_t)n_sm * kPeakThreads, st));
  cudaError_t e = cudaMallocAsync(&cyc_dev, sizeof(long long) * n_sm, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(sink, st);
    return cuda_error(e, "cudaMallocAsync");
  }
  std::vector<long long> cyc(n_sm);
  double r[PK_COUNT] = {};
#define NLOS_PK(K) \
  if (e == cudaSuccess) e = run_one<K>(n_sm, sink, cyc_dev, cyc, st, r[K]);
  NLOS_PK(PK_FFMA) NLOS_PK(PK_FFMA2) NLOS_PK(PK_SQRT) NLOS_PK(PK_RCP) NLOS_PK(PK_RSQRT)
  NLOS_PK(PK_LDS128) NLOS_PK(PK_RED_F32) NLOS_PK(PK_RED_U32) NLOS_PK(PK_RED_U64)
  NLOS_PK(PK_RMW_F32) NLOS_PK(PK_RED_F32_Q) NLOS_PK(PK_RED_U32_Q) NLOS_PK(PK_DFMA)
  NLOS_PK(PK_ATOM_F32)
#undef NLOS_PK
  cudaFreeAsync(sink, st);
  cudaFreeAsync(cyc_dev, st);
  if (e != cudaSuccess) return cuda_error(e, "nlos_measure_peaks");
  NLOS_CUDA_TRY(cudaStreamSynchronize(st));
  out->num_sms = n_sm;
  out->ffma = r[PK_FFMA];
  out->ffma2 = r[PK_FFMA2];
  out->sqrt_approx = r[PK_SQRT];
  out->rcp_approx = r[PK_RCP];
  out->rsqrt_approx = r[PK_RSQRT];
  out->lds128_broadcast = r[PK_LDS128];
  out->red_f32 = r[PK_RED_F32];
  out->red_u32 = r[PK_RED_U32];
  out->red_u64 = r[PK_RED_U64];
  out->rmw_f32 = r[PK_RMW_F32];
  out->red_f32_quarter = r[PK_RED_F32_Q];
  out->red_u32_quarter = r[PK_RED_U32_Q];
  out->dfma = r[PK_DFMA];
  out->atom_f32 = r[PK_ATOM_F32];
  return NLOS_OK;
}
