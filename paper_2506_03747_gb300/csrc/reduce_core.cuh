// Per-transient sums of the cube reductions (energy, and the cube's sum and
// sum of squares for the noise scale of Eq. 18/19), shared by nlos_reduce and
// nlos_reduce_static so that both give the same per-transient results.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nlos {

// Knuth's error-free sum: s + e == a + b exactly (round to nearest; the
// explicit intrinsics keep the compiler from reassociating or contracting).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Adds x and x^2 to the lane's sums, each kept as an unevaluated FP32 pair
// (hi + lo): the rounding error of every addition, and of the square (an
// fma recovers it exactly), goes to lo. So the lane sums are the FP64-quality
// sums of its bins, using the FP32 pipe; the FP64 pipe, which this GPU runs
// at a small fraction of its FP32 rate, only combines the lanes.
__device__ __forceinline__ void df_add(float x, float& sh, float& sl, float& qh, float& ql) {
  float s, e;
  two_sum(sh, x, s, e);
  sh = s;
  sl = __fadd_rn(sl, e);
  const float p = __fmul_rn(x, x);
  const float pe = __fmaf_rn(x, x, -p);  // x^2 - p, exactly
  two_sum(qh, p, s, e);
  qh = s;
  ql = __fadd_rn(ql, __fadd_rn(e, pe));
}

// (ah, al) += (bh, bl) for unevaluated FP32 pairs: the error-free sum of the
// high parts, the low parts and that sum's error added, then renormalised
// (|lo| <= half an ulp of hi), so a pair keeps about 48 bits.
__device__ __forceinline__ void df_add_pair(float& ah, float& al, float bh, float bl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  ah = __fadd_rn(s, e);
  al = __fsub_rn(e, __fsub_rn(ah, s));
}

// One warp's sums over a transient row of B bins (every lane returns the
// warp's values): the FP64 sum and sum of squares of the FP32 bins (lane
// sums as above, combined over the lanes by a fixed shuffle tree of pair
// additions, and converted to FP64 once) and the maximum.
__device__ __forceinline__ void trace_sums(const float* __restrict__ row, uint32_t B, int lane,
                                           double& s_out, double& q_out, float& m_out) {
  float sh = 0.f, sl = 0.f, qh = 0.f, ql = 0.f;
  float m = 0.0f;
  if ((B & 3u) == 0u) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
    for (uint32_t i = lane; i < B / 4; i += 32) {
      const float4 v = __ldg(r4 + i);
      df_add(v.x, sh, sl, qh, ql);
      df_add(v.y, sh, sl, qh, ql);
      df_add(v.z, sh, sl, qh, ql);
      df_add(v.w, sh, sl, qh, ql);
      m = fmaxf(m, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
    }
  } else {
    for (uint32_t i = lane; i < B; i += 32) {
      const float v = __ldg(row + i);
      df_add(v, sh, sl, qh, ql);
      m = fmaxf(m, v);
    }
  }
  // renormalise the lane pairs (lo accumulated plain roundings)
  {
    float t = __fadd_rn(sh, sl);
    sl = __fsub_rn(sl, __fsub_rn(t, sh));
    sh = t;
    t = __fadd_rn(qh, ql);
    ql = __fsub_rn(ql, __fsub_rn(t, qh));
    qh = t;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bsh = __shfl_xor_sync(0xffffffffu, sh, o);
    const float bsl = __shfl_xor_sync(0xffffffffu, sl, o);
    const float bqh = __shfl_xor_sync(0xffffffffu, qh, o);
    const float bql = __shfl_xor_sync(0xffffffffu, ql, o);
    df_add_pair(sh, sl, bsh, bsl);
    df_add_pair(qh, ql, bqh, bql);
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  s_out = (double)sh + (double)sl;
  q_out = (double)qh + (double)ql;
  m_out = m;
}

}  // namespace nlos
