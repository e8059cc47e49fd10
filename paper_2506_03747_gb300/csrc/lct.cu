// The paper's FFT forward model (the light-cone-transform convolution of the
// Theory section, Algorithm 1 steps 1.1-2.2) for an N x N confocal depth map
// with M time bins (N, M powers of two):
//   tau = R_t^{-1} F^{-1}[ F(R_z V) . F(PSF) ]
// on a zero-padded (2N) x (2N) x (2M) grid.
//
// Readings (as in the oracle): V holds albedo at depth bin D[x, y]; R_z maps
// depth bin j (1-based) to squared-depth sample ceil(j^2 / M) with weight
// 1 / (j M^2) (the perfect-square rows of the printed fine matrix, averaged
// over log2 M levels of (1/2) S_k); R_t^{-1} reads time bin j from sample
// ceil(j^2 / M) with weight M / j^4 (the v^{-3/2} factor that Eq. 3 implies);
// the PSF has one node per (x, y) column, the z node nearest
// (4 slope)^2 (x^2 + y^2), slope = w / (M c dt), circularly shifted so that
// node (N, N, M) is the origin.
//
// Arithmetic: FP64 throughout. The time resampling weights the earliest bins
// by up to M / 1 against M / j^4 at the signal, so FP32 round-off of the
// transforms (1e-7 of the largest value) would exceed the signal there.
//
// Layout: the work volume is [2N][2N][2M] complex (time fastest); each 1-D
// transform runs in shared memory (bit-reversed load, log2 L radix-2
// stages); along x and y a CTA takes several lines adjacent in time so that
// its loads and stores are coalesced.
#include "common.cuh"

#include <cmath>
#include <new>
#include <vector>

namespace nlos {
namespace {

constexpr int kFftThreads = 256;
constexpr size_t kFftSmem = 64 * 1024;  // bytes of lines per CTA

struct LctDims {
  uint32_t N, M;   // depth map side, bins
  uint32_t n2, m2; // 2N, 2M
};

// Lines of length L along one axis of the [2N][2N][2M] volume: line
// (o, i) starts at o * outer_stride + i (i < n_inner, consecutive in memory)
// and its samples are s_stride apart. A CTA takes T lines (o, i0..i0+T-1).
struct FftArgs {
  double2* data;
  const double2* tw;  // exp(-2 pi i k / Lmax), k < Lmax / 2
  uint32_t L, log2L, T, tw_step;
  uint64_t s_stride, outer_stride, n_inner;
  int inverse;         // conjugate twiddles and scale by 1 / L
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(kFftThreads) fft_lines_kernel(const FftArgs a) {
  extern __shared__ double2 buf[];  // [T][L]
  const uint64_t groups_per_outer = (a.n_inner + a.T - 1) / a.T;
  const uint64_t o = blockIdx.x / groups_per_outer;
  const uint64_t i0 = (blockIdx.x % groups_per_outer) * a.T;
  const uint32_t nl = (uint32_t)min((uint64_t)a.T, a.n_inner - i0);
  const uint64_t base = o * a.outer_stride + i0;
  // load, bit-reversed within each line; consecutive threads take
  // consecutive lines of one sample (coalesced when s_stride > 1)
  for (uint32_t e = threadIdx.x; e < a.L * nl; e += blockDim.x) {
    const uint32_t s = a.s_stride == 1 ? e % a.L : e / nl;
    const uint32_t l = a.s_stride == 1 ? e / a.L : e % nl;
    const uint32_t r = __brev(s) >> (32 - a.log2L);
    buf[l * a.L + r] = a.data[base + l + (uint64_t)s * a.s_stride];
  }
  __syncthreads();
  const uint32_t half = a.L / 2;
  for (uint32_t m = 1; m < a.L; m <<= 1) {
    const uint32_t step = (a.L / (2 * m)) * a.tw_step;  // twiddle index stride
    for (uint32_t b = threadIdx.x; b < half * nl; b += blockDim.x) {
      const uint32_t l = b / half, k = b % half;
      const uint32_t j = k % m;
      const uint32_t i1 = (k / m) * 2 * m + j, i2 = i1 + m;
      double2 w = a.tw[j * step];
      if (a.inverse) w.y = -w.y;
      double2* line = buf + l * a.L;
      const double2 x = line[i1];
      const double2 y = cmul(w, line[i2]);
      line[i1] = make_double2(x.x + y.x, x.y + y.y);
      line[i2] = make_double2(x.x - y.x, x.y - y.y);
    }
    __syncthreads();
  }
  const double sc = a.inverse ? 1.0 / (double)a.L : 1.0;
  for (uint32_t e = threadIdx.x; e < a.L * nl; e += blockDim.x) {
    const uint32_t s = a.s_stride == 1 ? e % a.L : e / nl;
    const uint32_t l = a.s_stride == 1 ? e / a.L : e % nl;
    const double2 v = buf[l * a.L + s];
    a.data[base + l + (uint64_t)s * a.s_stride] = make_double2(v.x * sc, v.y * sc);
  }
}

// PSF (reading above) written circularly shifted into a zeroed volume.
__global__ void psf_kernel(double2* vol, LctDims d, double slope4sq) {
  const uint64_t col = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= (uint64_t)d.n2 * d.n2) return;
  const uint32_t i = (uint32_t)(col / d.n2), j = (uint32_t)(col % d.n2);
  const double x = -1.0 + 2.0 * i / (double)(d.n2 - 1);
  const double y = -1.0 + 2.0 * j / (double)(d.n2 - 1);
  const double dz = 2.0 / (double)(d.m2 - 1);
  const double target = slope4sq * (x * x + y * y);
  const double kf = rint((target + 1.0) / dz);
  if (!(kf >= 0.0 && kf < (double)d.m2)) return;
  const int64_t k = (int64_t)kf;
  if (fabs(target - (-1.0 + (double)k * dz)) > 0.5 * dz + 1e-12) return;
  const uint32_t is = (i + d.N) % d.n2;  // origin at node (N, N, M)
  const uint32_t js = (j + d.N) % d.n2;
  const uint32_t ks = (uint32_t)((k + d.M) % d.m2);
  vol[((uint64_t)is * d.n2 + js) * d.m2 + ks] = make_double2(1.0, 0.0);
}

// R_z V into the zeroed volume: one voxel per depth-map pixel.
__global__ void volume_kernel(double2* vol, LctDims d, const int32_t* depth, const float* albedo) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N * d.N) return;
  const uint32_t x = p / d.N, y = p % d.N;
  const int32_t z = depth[p];
  if (z < 0 || z >= (int32_t)d.M) return;
  const uint64_t j = (uint64_t)z + 1;
  const uint64_t r = (j * j + d.M - 1) / d.M - 1;
  const double a = albedo ? (double)albedo[p] : 0.5;
  vol[((uint64_t)x * d.n2 + y) * d.m2 + r] =
      make_double2(a / ((double)j * d.M * d.M), 0.0);
}

__global__ void multiply_kernel(double2* vol, const double2* psf_hat, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    vol[i] = cmul(vol[i], psf_hat[i]);
}

// Crop to N x N x M and resample time: tau[x][y][j - 1] = Re W[x][y][r(j)] M / j^4.
__global__ void time_kernel(const double2* vol, LctDims d, float* tau) {
  const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (uint64_t)d.N * d.N * d.M) return;
  const uint64_t p = e / d.M;
  const uint64_t j = e % d.M + 1;
  const uint64_t x = p / d.N, y = p % d.N;
  const uint64_t r = (j * j + d.M - 1) / d.M - 1;
  const double jd = (double)j;
  tau[e] = (float)(vol[(x * d.n2 + y) * d.m2 + r].x * ((double)d.M / (jd * jd * jd * jd)));
}

bool pow2(uint32_t v) { return v >= 2 && (v & (v - 1)) == 0; }
uint32_t ilog2(uint32_t v) {
  uint32_t r = 0;
  while ((1u << r) < v) ++r;
  return r;
}

}  // namespace
}  // namespace nlos

struct nlos_lct {
  nlos::LctDims d;
  double2* work = nullptr;
  double2* psf_hat = nullptr;
  double2* tw = nullptr;
  uint32_t lmax = 0;
  int device = 0;
};

namespace nlos {
namespace {

cudaError_t fft3(const nlos_lct& p, double2* vol, int inverse, cudaStream_t st) {
  const LctDims& d = p.d;
  struct Axis {
    uint32_t L;
    uint64_t s_stride, outer_stride, n_inner, n_outer;
  };
  const uint64_t m2 = d.m2, n2 = d.n2;
  const Axis axes[3] = {
      {d.m2, 1, m2, 1, n2 * n2},             // time: contiguous lines
      {d.n2, m2, n2 * m2, m2, n2},           // y: lines (x, t)
      {d.n2, n2 * m2, m2, m2, n2},           // x: lines (y, t)
  };
  for (const Axis& ax : axes) {
    FftArgs a;
    a.data = vol;
    a.tw = p.tw;
    a.L = ax.L;
    a.log2L = ilog2(ax.L);
    a.tw_step = p.lmax / ax.L;
    a.s_stride = ax.s_stride;
    a.outer_stride = ax.outer_stride;
    a.n_inner = ax.n_inner;
    a.inverse = inverse;
    const size_t line_bytes = sizeof(double2) * ax.L;
    uint32_t T = ax.s_stride == 1 ? 1u : (uint32_t)std::max<size_t>(1, kFftSmem / line_bytes);
    if (T > 16) T = 16;
    if (ax.s_stride == 1) {
      // contiguous lines: each line is its own "outer" index of one line
      a.n_inner = 1;
      a.outer_stride = ax.L;
    }
    a.T = T;
    const uint64_t groups = (a.n_inner + T - 1) / T;
    const uint64_t blocks = (ax.s_stride == 1 ? ax.n_outer : ax.n_outer) * groups;
    const size_t smem = line_bytes * T;
    cudaError_t e = cudaFuncSetAttribute(fft_lines_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    fft_lines_kernel<<<(unsigned)blocks, kFftThreads, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace
}  // namespace nlos

using namespace nlos;

extern "C" {

nlos_status nlos_lct_create(uint32_t n, uint32_t m, double wall_half_m, double bin_width_s,
                            void* cuda_stream, nlos_lct** out) {
  clear_error();
  if (!out) return set_error(NLOS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!pow2(n) || !pow2(m) || n > 1024 || m > 4096)
    return set_error(NLOS_EINVAL, "n and m must be powers of two, 2 <= n <= 1024, 2 <= m <= 4096");
  if (!(std::isfinite(wall_half_m) && wall_half_m > 0 && std::isfinite(bin_width_s) && bin_width_s > 0))
    return set_error(NLOS_EINVAL, "wall_half_m and bin_width_s must be finite and > 0");
  nlos_lct* p = new (std::nothrow) nlos_lct();
  if (!p) return set_error(NLOS_ENOMEM, "host allocation failed");
  p->d = LctDims{n, m, 2 * n, 2 * m};
  p->lmax = std::max(2 * n, 2 * m);
  const uint64_t nvol = (uint64_t)p->d.n2 * p->d.n2 * p->d.m2;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  auto fail = [&](cudaError_t e, const char* what) {
    if (p->work) cudaFree(p->work);
    if (p->psf_hat) cudaFree(p->psf_hat);
    if (p->tw) cudaFree(p->tw);
    delete p;
    return cuda_error(e, what);
  };
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) return fail(e, "cudaGetDevice");
  if ((e = cudaMalloc(&p->work, sizeof(double2) * nvol)) != cudaSuccess ||
      (e = cudaMalloc(&p->psf_hat, sizeof(double2) * nvol)) != cudaSuccess ||
      (e = cudaMalloc(&p->tw, sizeof(double2) * (p->lmax / 2))) != cudaSuccess)
    return fail(e, "cudaMalloc");
  std::vector<double2> tw(p->lmax / 2);
  const double pi = 3.14159265358979323846;
  for (uint32_t k = 0; k < p->lmax / 2; ++k) {
    const double ang = -2.0 * pi * (double)k / (double)p->lmax;
    tw[k] = make_double2(std::cos(ang), std::sin(ang));
  }
  if ((e = cudaMemcpyAsync(p->tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess ||
      (e = cudaMemsetAsync(p->psf_hat, 0, sizeof(double2) * nvol, st)) != cudaSuccess)
    return fail(e, "cudaMemcpyAsync");
  const double slope = wall_half_m / ((double)m * kLightSpeed * bin_width_s);
  const uint64_t cols = (uint64_t)p->d.n2 * p->d.n2;
  psf_kernel<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(p->psf_hat, p->d, 16.0 * slope * slope);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "psf_kernel");
  if ((e = fft3(*p, p->psf_hat, 0, st)) != cudaSuccess) return fail(e, "fft");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e, "cudaStreamSynchronize");
  *out = p;
  return NLOS_OK;
}

nlos_status nlos_lct_forward(nlos_lct* plan, const int32_t* depth_dev, const float* albedo_dev,
                             float* tau_dev, void* cuda_stream) {
  clear_error();
  if (!plan || !depth_dev || !tau_dev)
    return set_error(NLOS_EINVAL, "plan, depth_dev and tau_dev must not be NULL");
  const LctDims& d = plan->d;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const uint64_t nvol = (uint64_t)d.n2 * d.n2 * d.m2;
  NLOS_CUDA_TRY(cudaMemsetAsync(plan->work, 0, sizeof(double2) * nvol, st));
  volume_kernel<<<(d.N * d.N + 255) / 256, 256, 0, st>>>(plan->work, d, depth_dev, albedo_dev);
  NLOS_CUDA_TRY(cudaGetLastError());
  NLOS_CUDA_TRY(fft3(*plan, plan->work, 0, st));
  multiply_kernel<<<2048, 256, 0, st>>>(plan->work, plan->psf_hat, nvol);
  NLOS_CUDA_TRY(cudaGetLastError());
  NLOS_CUDA_TRY(fft3(*plan, plan->work, 1, st));
  const uint64_t n_out = (uint64_t)d.N * d.N * d.M;
  time_kernel<<<(unsigned)((n_out + 255) / 256), 256, 0, st>>>(plan->work, d, tau_dev);
  NLOS_CUDA_TRY(cudaGetLastError());
  return NLOS_OK;
}

nlos_status nlos_lct_destroy(nlos_lct* plan) {
  clear_error();
  if (!plan) return set_error(NLOS_EINVAL, "plan is NULL");
  cudaDeviceSynchronize();
  cudaFree(plan->work);
  cudaFree(plan->psf_hat);
  cudaFree(plan->tw);
  delete plan;
  return NLOS_OK;
}

}  // extern "C"
