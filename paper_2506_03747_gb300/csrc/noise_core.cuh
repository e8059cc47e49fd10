// Device Poisson noise of the GB300 NLOS simulator (Eq. 18/19 of arXiv
// 2506.03747, Algorithm 1 step 2.4): Philox4x32-10 draws and the inversion /
// PTRS samplers. Shared by the standalone noise kernel and the
// persistent serving kernel.
#pragma once

#include "common.cuh"
#include "device_util.cuh"

namespace nlos {

// ---------------------------------------------------------------------------
// Poisson sampling, step for step as the CPU oracle so that both take every
// integer decision in the same precision: single-precision lambda, uniforms
// and inversion sums, PTRS in double (explicit __d*_rn / __f*_rn intrinsics
// keep the compiler from contracting into FMAs).
// Draws (key = (seed_lo, seed_hi)): bins go in groups of four, g = index / 4;
// the first uniform of a bin is word (index mod 4) of the block at counter
// (g_lo, g_hi, 0, tag), so one Philox block serves four bins' first draws;
// further uniforms come from the bin's own stream at counters
// (index_lo, index_hi, 1 + j, tag). A word w gives ((w >> 9) + 0.5) * 2^-23.
//  * lambda < 30: inversion by sequential search from the first uniform:
//    p_0 = expf(-lambda), p_k = (p_{k-1} lambda) (1/k), F_k = F_{k-1} + p_k,
//    count = first k with u <= F_k (or the first k whose term leaves F
//    unchanged, or 1000);
//  * 30 <= lambda < 150: the sum of ceil(lambda / 30) inversion draws of mean
//    lambda / ceil(lambda / 30), the first from the first uniform and the
//    others from the own stream (exact: a sum of independent Poisson
//    variables is Poisson);
//  * lambda >= 150: Hoermann's PTRS (1993), transformed rejection with
//    squeeze, in double, on the own stream.
// ---------------------------------------------------------------------------
// All three are exact; the inversion takes one uniform and about lambda
// multiply-adds, where Knuth's product method takes about lambda uniforms.
constexpr float kInvMax = 30.0f;
constexpr float kSplitMax = 150.0f;
constexpr int kRcpTable = 64;  // 1/k for k < kRcpTable from a table (shared memory)

__device__ __forceinline__ float word_uniform(uint32_t w) {
  return __fmul_rn(__fadd_rn((float)(w >> 9), 0.5f), 0x1p-23f);
}

// The Philox block of group g (the first draws of bins 4g .. 4g + 3).
__device__ __forceinline__ uint4 group_block(uint64_t g, uint64_t seed, uint32_t tag) {
  return philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), 0u, tag), (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t group_word(const uint4& b, uint32_t r) {
  return r == 0 ? b.x : r == 1 ? b.y : r == 2 ? b.z : b.w;
}

// A bin's own stream (blocks 1, 2, ... of its counter), computed on first use.
struct BinStream {
  uint4 ctr;
  uint32_t k0, k1;
  uint4 buf;
  int pos;
  __device__ BinStream(uint64_t index, uint64_t seed, uint32_t tag) {
    ctr = make_uint4((uint32_t)index, (uint32_t)(index >> 32), 0u, tag);
    k0 = (uint32_t)seed;
    k1 = (uint32_t)(seed >> 32);
    pos = 4;
  }
  __device__ __forceinline__ float uniform() {
    if (pos == 4) {
      ctr.z += 1u;
      buf = philox4x32_10(ctr, k0, k1);
      pos = 0;
    }
    const uint32_t w = pos == 0 ? buf.x : pos == 1 ? buf.y : pos == 2 ? buf.z : buf.w;
    ++pos;
    return word_uniform(w);
  }
};

// 1/k rounded to single precision (the correctly rounded reciprocal, as the
// host's 1.0f / k); rcp: a table of kRcpTable entries or null.
__device__ __forceinline__ float recip_k(uint32_t k, const float* rcp) {
  return (rcp && k < (uint32_t)kRcpTable) ? rcp[k] : __frcp_rn((float)k);
}

__device__ __forceinline__ uint32_t poisson_inversion(float lam, float u, const float* rcp) {
  float p = expf(-lam);
  float F = p;
  uint32_t k = 0;
  while (u > F && k < 1000u) {
    k += 1u;
    p = __fmul_rn(__fmul_rn(p, lam), recip_k(k, rcp));
    const float Fn = __fadd_rn(F, p);
    if (Fn == F) break;
    F = Fn;
  }
  return k;
}

__device__ __forceinline__ uint32_t poisson_ptrs(float lam_f, BinStream& st) {
  const double lam = (double)lam_f;
  const double slam = sqrt(lam);
  const double loglam = log(lam);
  const double b = __dadd_rn(0.931, __dmul_rn(2.53, slam));
  const double a = __dadd_rn(-0.059, __dmul_rn(0.02483, b));
  const double inv_alpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dsub_rn(b, 3.4)));
  const double v_r = __dsub_rn(0.9277, __ddiv_rn(3.6224, __dsub_rn(b, 2.0)));
  for (int it = 0; it < 1000; ++it) {
    const double U = __dsub_rn((double)st.uniform(), 0.5);
    const double V = (double)st.uniform();
    const double us = __dsub_rn(0.5, fabs(U));
    const double kf = floor(__dadd_rn(
        __dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(2.0, a), us), b), U), lam), 0.43));
    if (us >= 0.07 && V <= v_r) return (uint32_t)kf;
    if (kf < 0.0 || (us < 0.013 && V > us)) continue;
    const double lhs = __dsub_rn(__dadd_rn(log(V), log(inv_alpha)),
                                 log(__dadd_rn(__ddiv_rn(a, __dmul_rn(us, us)), b)));
    const double rhs =
        __dsub_rn(__dadd_rn(-lam, __dmul_rn(kf, loglam)), lgamma(__dadd_rn(kf, 1.0)));
    if (lhs <= rhs) return (uint32_t)kf;
  }
  return (uint32_t)floor(lam);
}

// lambda >= 30, out of line: these bins are rare (the bright bins of a
// cube), and inlined their paths would set the register budget of every bin.
static __device__ __noinline__ uint32_t poisson_large(float lam, float u0, uint64_t index,
                                                      uint64_t seed, uint32_t tag,
                                                      const float* rcp) {
  BinStream st(index, seed, tag);
  if (lam < kSplitMax) {
    const float parts = ceilf(__fdiv_rn(lam, kInvMax));
    const float sub = __fdiv_rn(lam, parts);
    uint32_t k = poisson_inversion(sub, u0, rcp);
    for (int i = 1; i < (int)parts; ++i) k += poisson_inversion(sub, st.uniform(), rcp);
    return k;
  }
  return poisson_ptrs(lam, st);
}

// The count of bin `index` given its first uniform u0 (from its group block).
__device__ __forceinline__ uint32_t poisson_from(float lam, float u0, uint64_t index,
                                                 uint64_t seed, uint32_t tag, const float* rcp) {
  if (!(lam > 0.0f)) return 0u;
  if (lam < kInvMax) return poisson_inversion(lam, u0, rcp);
  return poisson_large(lam, u0, index, seed, tag, rcp);
}

// One bin on its own (its group block is computed for it alone).
__device__ __forceinline__ uint32_t poisson_sample(float lam, uint64_t index, uint64_t seed,
                                                   uint32_t tag, const float* rcp = nullptr) {
  if (!(lam > 0.0f)) return 0u;
  const uint4 b = group_block(index >> 2, seed, tag);
  return poisson_from(lam, word_uniform(group_word(b, (uint32_t)(index & 3u))), index, seed, tag,
                      rcp);
}

// Fills a shared table of 1/k (k < kRcpTable; entry 0 unused) with nthreads
// threads starting at thread t0; the caller synchronises before use.
__device__ __forceinline__ void fill_rcp_table(float* rcp, int t, int nthreads) {
  for (int k = t; k < kRcpTable; k += nthreads) rcp[k] = k ? __frcp_rn((float)k) : 0.0f;
}

// Counts of the bins [b, e) of a cube part (local indices; the global index
// of local bin l is index_base + l, and lambda = scale * tau + dark), group by
// group: this thread takes the groups gb + j0, gb + j0 + stride, ... of the
// groups of four global indices that meet [b, e), computes each group's
// Philox block once, and samples its (up to four) bins of the range. Interior
// groups of an aligned part load and store four bins at a time.
// DEFER: bins with lambda >= 30 get kDeferredCount instead of their count and
// are listed (DeferList); a second pass samples them (noise_deferred_bin for
// the dense list, noise_deferred_warp for overflowed regions), so the first
// pass holds no out-of-line call and keeps its registers for the common bins.
constexpr uint32_t kDeferredCount = 0xFFFFFFFFu;

// Where DEFER puts the deferred bins: a dense list of their local indices
// (count in hdr[0], at most cap entries) and, for a warp whose bins no longer
// fit, the first group of its 32-group region (count in hdr[1]); the lanes of
// a warp take consecutive groups (j0 = 32 * warp + lane, stride a multiple of
// 32), so the lanes still in the loop are always a prefix of the warp.
struct DeferList {
  unsigned long long* hdr;       // [2]: dense entries claimed, regions listed
  uint32_t* bins;                // [cap] local bin indices (kDeferredCount: skip)
  unsigned long long* regions;   // first groups of overflowed warp regions
  uint32_t cap;
};

template <bool DEFER = false>
__device__ __forceinline__ void noise_groups(const float* __restrict__ tau,
                                             uint32_t* __restrict__ counts, uint64_t b, uint64_t e,
                                             uint64_t index_base, float scale, float dark,
                                             uint64_t seed, uint32_t tag, const float* rcp,
                                             uint64_t j0, uint64_t stride,
                                             const DeferList* dl = nullptr) {
  if (b >= e) return;
  const uint64_t gb = (index_base + b) >> 2, ge = (index_base + e + 3) >> 2;
  const bool vec_ok = ((((uintptr_t)tau) | ((uintptr_t)counts)) & 15u) == 0;
  for (uint64_t g = gb + j0; g < ge; g += stride) {
    const int64_t l0 = (int64_t)(4 * g) - (int64_t)index_base;  // local index of bin 4g
    const bool vec = vec_ok && (l0 & 3) == 0 && l0 >= (int64_t)b && l0 + 4 <= (int64_t)e;
    float t[4];
    uint32_t in = 0xFu;  // bit r: bin 4g + r lies in the range
    if (vec) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(tau + l0));
      t[0] = v.x; t[1] = v.y; t[2] = v.z; t[3] = v.w;
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int64_t l = l0 + r;
        const bool ok = l >= (int64_t)b && l < (int64_t)e;
        t[r] = ok ? __ldg(tau + l) : 0.0f;
        if (!ok) in &= ~(1u << r);
      }
    }
    const uint4 blk = group_block(g, seed, tag);
    uint32_t c[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      // bins outside the range are not sampled
      const float lam = ((in >> r) & 1u) ? fmaf(scale, t[r], dark) : 0.0f;
      const float u0 = word_uniform(group_word(blk, (uint32_t)r));
      if (DEFER)
        c[r] = !(lam > 0.0f) ? 0u
               : lam < kInvMax ? poisson_inversion(lam, u0, rcp)
                               : kDeferredCount;
      else
        c[r] = poisson_from(lam, u0, 4 * g + r, seed, tag, rcp);
    }
    if (DEFER) {
      uint32_t dm = 0;  // bit r: bin 4g + r was deferred
#pragma unroll
      for (int r = 0; r < 4; ++r) dm |= (uint32_t)(c[r] == kDeferredCount) << r;
      const uint32_t act = __activemask();
      if (__any_sync(act, dm != 0u)) {
        const uint32_t lane = threadIdx.x & 31u;
        const uint32_t cnt = (uint32_t)__popc(dm);
        uint32_t incl = cnt;  // inclusive prefix sum over the lanes (a prefix of the warp)
#pragma unroll
        for (uint32_t o = 1; o < 32u; o <<= 1) {
          const uint32_t v = __shfl_up_sync(act, incl, o);
          if (lane >= o) incl += v;
        }
        const uint32_t total = __shfl_sync(act, incl, 31 - __clz((int)act));
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&dl->hdr[0], (unsigned long long)total);
        base = __shfl_sync(act, base, 0);
        const unsigned long long o0 = base + incl - cnt;
        const bool fits = base + total <= dl->cap;  // the same in every lane
        uint32_t o = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if ((dm >> r) & 1u) {
            const unsigned long long slot = o0 + o++;
            if (slot < dl->cap) dl->bins[slot] = fits ? (uint32_t)(l0 + r) : kDeferredCount;
          }
        if (!fits && lane == 0) {
          const unsigned long long k = atomicAdd(&dl->hdr[1], 1ull);
          dl->regions[k] = g - lane;  // the warp region's first group
        }
      }
    }
    if (vec) {
      *reinterpret_cast<uint4*>(counts + l0) = make_uint4(c[0], c[1], c[2], c[3]);
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int64_t l = l0 + r;
        if (l >= (int64_t)b && l < (int64_t)e) counts[l] = c[r];
      }
    }
  }
}

// Second pass, one deferred bin (local index l): the count with the bin's
// first-pass draws (its group word and its own stream).
__device__ __forceinline__ void noise_deferred_bin(const float* __restrict__ tau,
                                                   uint32_t* __restrict__ counts, uint64_t l,
                                                   uint64_t index_base, float scale, float dark,
                                                   uint64_t seed, uint32_t tag, const float* rcp) {
  const uint64_t i = index_base + l;
  const float lam = fmaf(scale, __ldg(tau + l), dark);
  const uint4 blk = group_block(i >> 2, seed, tag);
  counts[l] = poisson_large(lam, word_uniform(group_word(blk, (uint32_t)(i & 3u))), i, seed, tag,
                            rcp);
}

// Second pass over one 32-group region (global bins 4 G0 .. 4 G0 + 127; local
// index l = global - index_base, inside [0, n)) by one warp: the bins the first
// pass marked kDeferredCount (lambda >= 30) are dealt out to the lanes, one bin
// a lane at a time, and sampled with the same draws (the bin's group word and
// its own stream), so bright runs of bins are searched side by side.
__device__ __forceinline__ void noise_deferred_warp(const float* __restrict__ tau,
                                                    uint32_t* __restrict__ counts, uint64_t n,
                                                    uint64_t G0, uint64_t index_base,
                                                    float scale, float dark, uint64_t seed,
                                                    uint32_t tag, const float* rcp) {
  const uint32_t lane = threadIdx.x & 31u;
  const int64_t w0 = (int64_t)(4 * G0) - (int64_t)index_base;
  uint32_t m[4];
  uint32_t total = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t l = w0 + 32 * r + (int64_t)lane;
    const bool d = l >= 0 && l < (int64_t)n && counts[l] == kDeferredCount;
    m[r] = __ballot_sync(0xffffffffu, d);
    total += (uint32_t)__popc(m[r]);
  }
  for (uint32_t base = 0; base < total; base += 32u) {
    uint32_t k = base + lane;  // this lane's deferred bin, in order
    if (k < total) {
      int r = 0;
      while (k >= (uint32_t)__popc(m[r])) {
        k -= (uint32_t)__popc(m[r]);
        ++r;
      }
      uint32_t mm = m[r];
      for (uint32_t j = 0; j < k; ++j) mm &= mm - 1u;  // drop the k lowest set bits
      const uint32_t src = (uint32_t)__ffs((int)mm) - 1u;
      const int64_t l = w0 + 32 * r + (int64_t)src;
      noise_deferred_bin(tau, counts, (uint64_t)l, index_base, scale, dark, seed, tag, rcp);
    }
  }
}

// Noise scale from a cube's reduction results (identical in every thread):
//  PEAK:     scale = peak_photons / max tau_G (0 for an empty cube);
//  PAPER_NR: scale = sigma_n = Var(tau_G) / 10^(nr/10), population variance
//            over the n bins of the whole cube.
__device__ __forceinline__ float noise_scale_of(float peak, double sum, double sumsq, int mode,
                                                float peak_photons, float nr_db, uint64_t n) {
  if (mode == NLOS_NOISE_PEAK) return peak > 0.0f ? __fdiv_rn(peak_photons, peak) : 0.0f;
  const double nn = (double)n;
  const double mean = sum / nn;
  double var = sumsq / nn - mean * mean;
  if (var < 0.0) var = 0.0;
  return (float)(var / pow(10.0, (double)nr_db / 10.0));
}

__device__ __forceinline__ float noise_scale_from(const SceneScratch* sc, int mode,
                                                  float peak_photons, float nr_db, uint64_t n) {
  return noise_scale_of(__uint_as_float(sc->peak_bits), sc->sum, sc->sumsq, mode, peak_photons,
                        nr_db, n);
}

}  // namespace nlos
