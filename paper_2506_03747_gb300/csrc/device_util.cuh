// Device helpers: mbarrier with bounded waits, TMA bulk copies, Philox4x32-10.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nlos {

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy (TMA) wrappers. All waits are bounded by a clock64
// deadline; a wait that gives up returns false and the caller records an
// error status instead of hanging the GPU.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Ends the barrier's use (no arrival or transaction may be pending); it can
// then be initialised again.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared (this CTA), completion signalled on bar.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// ~1 s at 2 GHz; a bulk copy from valid global memory completes in microseconds.
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Fire-and-forget atomics.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_add_shared(uint32_t addr, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// red.shared.add.f32 [addr], v  if  bin < lim (unsigned)  [and cn > 0]:
// the predicate is formed and applied inside one asm block, so no branch.
__device__ __forceinline__ void red_add_shared_if_bin(uint32_t addr, float v, uint32_t bin,
                                                      uint32_t lim) {
  asm volatile(
      "{\n .reg .pred p;\n setp.lt.u32 p, %2, %3;\n @p red.shared.add.f32 [%0], %1;\n}\n" ::"r"(addr),
      "f"(v), "r"(bin), "r"(lim)
      : "memory");
}

__device__ __forceinline__ void red_add_shared_if_bin_cos(uint32_t addr, float v, uint32_t bin,
                                                          uint32_t lim, float cn) {
  asm volatile(
      "{\n .reg .pred p, q;\n setp.lt.u32 p, %2, %3;\n setp.gt.and.f32 q, %4, 0f00000000, p;\n"
      " @q red.shared.add.f32 [%0], %1;\n}\n" ::"r"(addr),
      "f"(v), "r"(bin), "r"(lim), "f"(cn)
      : "memory");
}

// Hardware reciprocal square root estimate (flush-to-zero; inputs here are
// squared distances, never subnormal).
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void red_add_global(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ void red_add_global_v4(float* p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11): ten rounds of
//   (c0, c1, c2, c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
// with the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct Philox {
  static constexpr uint32_t M0 = 0xD2511F53u;
  static constexpr uint32_t M1 = 0xCD9E8D57u;
  static constexpr uint32_t W0 = 0x9E3779B9u;
  static constexpr uint32_t W1 = 0xBB67AE85u;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += Philox::W0;
      k1 += Philox::W1;
    }
    uint32_t lo0 = Philox::M0 * c.x;
    uint32_t hi0 = __umulhi(Philox::M0, c.x);
    uint32_t lo1 = Philox::M1 * c.z;
    uint32_t hi1 = __umulhi(Philox::M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

}  // namespace nlos
