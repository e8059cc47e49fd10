// Device Poisson noise of the GB300 NLOS simulator (Eq. 18/19 of arXiv
// 2506.03747, Algorithm 1 step 2.4): per-bin Philox4x32-10 streams and the
// Knuth / PTRS samplers. Shared by the standalone noise kernel and the
// persistent serving kernel.
#pragma once

#include "common.cuh"
#include "device_util.cuh"

namespace nlos {

// ---------------------------------------------------------------------------
// Poisson sampling, step for step as the CPU oracle so that both take every
// integer decision in the same precision: single-precision lambda, uniforms
// and Knuth threshold, PTRS in double (explicit __d*_rn / __f*_rn intrinsics
// keep the compiler from contracting into FMAs).
// Per-bin stream: key = (seed_lo, seed_hi), counter = (index_lo, index_hi,
// block, stream_tag); a word w gives the uniform ((w >> 9) + 0.5) * 2^-23.
//  * lambda < 30: Knuth's multiplication method against expf(-lambda);
//  * 30 <= lambda < 150: the sum of ceil(lambda / 30) Knuth draws of mean
//    lambda / ceil(lambda / 30), one after the other from the same stream
//    (exact: a sum of independent Poisson variables is Poisson);
//  * lambda >= 150: Hoermann's PTRS (1993), transformed rejection with
//    squeeze, in double.
// ---------------------------------------------------------------------------
// All three are exact; the split only moves work between Knuth's single-
// precision products (about lambda of them) and the PTRS branch, which runs
// in FP64 (64 times slower per instruction on this part than FP32).
constexpr float kKnuthMax = 30.0f;
constexpr float kSplitMax = 150.0f;

struct BinStream {
  uint4 ctr;
  uint32_t k0, k1;
  uint4 buf;
  int pos;
  __device__ BinStream(uint64_t index, uint64_t seed, uint32_t tag) {
    ctr = make_uint4((uint32_t)index, (uint32_t)(index >> 32), 0u, tag);
    k0 = (uint32_t)seed;
    k1 = (uint32_t)(seed >> 32);
    buf = philox4x32_10(ctr, k0, k1);
    pos = 0;
  }
  __device__ __forceinline__ float uniform() {
    if (pos == 4) {
      ctr.z += 1u;
      buf = philox4x32_10(ctr, k0, k1);
      pos = 0;
    }
    const uint32_t w = pos == 0 ? buf.x : pos == 1 ? buf.y : pos == 2 ? buf.z : buf.w;
    ++pos;
    return __fmul_rn(__fadd_rn((float)(w >> 9), 0.5f), 0x1p-23f);
  }
};

__device__ inline uint32_t poisson_knuth(float lam, BinStream& st) {
  const float limit = expf(-lam);
  float prod = 1.0f;
  uint32_t k = 0;
  for (int it = 0; it < 1000; ++it) {
    prod = __fmul_rn(prod, st.uniform());
    if (prod <= limit) return k;
    k += 1;
  }
  return k;
}

// Out of line: the PTRS range is rare (lambda >= 150), and inlined it would
// set the register budget of every bin's path. The stream is passed by value
// (it is the bin's last sampler), so it stays in registers on both sides.
static __device__ __noinline__ uint32_t poisson_ptrs(float lam_f, BinStream st) {
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

__device__ __forceinline__ uint32_t poisson_sample(float lam, uint64_t index, uint64_t seed,
                                                   uint32_t tag) {
  if (!(lam > 0.0f)) return 0u;
  BinStream st(index, seed, tag);
  if (lam < kKnuthMax) return poisson_knuth(lam, st);
  if (lam < kSplitMax) {
    const float parts = ceilf(__fdiv_rn(lam, kKnuthMax));
    const float sub = __fdiv_rn(lam, parts);
    uint32_t k = 0;
    for (int i = 0; i < (int)parts; ++i) k += poisson_knuth(sub, st);
    return k;
  }
  return poisson_ptrs(lam, st);
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
