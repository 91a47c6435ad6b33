// Kernels of the inversion loop around the gradient (Sec. 2.3 and the
// imaging experiments of Sec. 3.2): the per-block low-pass of wavelets and
// traces, gathered by shot, and the gradient-descent update of the sound
// speed.  Both are HBM-bound elementwise / short-convolution passes that run
// once per iteration, next to the two propagations of every shot.
//
// Low-pass: one CTA filters a segment of LP_TILE samples of one row.  The
// segment plus M samples on each side is staged in shared memory (zeros
// outside the record), the 2M+1 taps are evaluated once per CTA, and each
// thread accumulates LP_PER_THREAD outputs over j = -M..M in that order.
//
// Update: two grid-stride passes.  The first reduces max |d| (d = dJ/dvp,
// masked) by an unsigned maximum over the bit patterns of |d|: the result is
// exact and independent of scheduling, and a NaN or Inf anywhere wins the
// maximum.  The second applies the normalised step with clipping; a
// non-finite maximum turns every vp into NaN, so that the next propagation
// reports the model as non-finite instead of clipping it silently.
#include "fwi.h"

#include <cuda_runtime.h>

#include <cmath>
#include <string>

namespace fwi {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int LP_THREADS = 256;
constexpr int LP_PER_THREAD = 4;
constexpr int LP_TILE = LP_THREADS * LP_PER_THREAD;
constexpr int LP_MAX_IDS = 512;   // ids per launch (kernel-parameter array)
constexpr double kPi = 3.14159265358979323846;

static_assert(FWI_LOWPASS_MAX_HALF_WIDTH <= 2048, "shared-memory staging assumes M <= 2048");

struct LowpassArgs {
  const float* in;
  float* out;
  long long nt;
  int rows;
  int M;
  float a;         // 2 f_max dt
  float inv_m1;    // 1 / (M + 1)
  float inv_norm;  // 1 / sum_j sinc(a j) w_j, evaluated on the host in double
  int ids[LP_MAX_IDS];
};

__global__ void __launch_bounds__(LP_THREADS) k_lowpass(const __grid_constant__ LowpassArgs p) {
  extern __shared__ float sm[];
  const int M = p.M;
  const int ntap = 2 * M + 1;
  float* taps = sm;
  float* xs = sm + ntap;   // xs[k] = x[t0 - M + k], k < LP_TILE + 2M
  const long long t0 = (long long)blockIdx.x * LP_TILE;
  const long long in_row = (long long)p.ids[blockIdx.z] * p.rows + blockIdx.y;
  const long long out_row = (long long)blockIdx.z * p.rows + blockIdx.y;
  const float* x = p.in + in_row * p.nt;

  for (int k = threadIdx.x; k < ntap; k += LP_THREADS) {
    const int j = k - M;
    const float arg = p.a * (float)j;
    const float s = (j == 0) ? 1.0f : sinpif(arg) / (3.14159265358979f * arg);
    const float w = 0.5f * (1.0f + cospif((float)j * p.inv_m1));
    taps[k] = s * w * p.inv_norm;
  }
  const int W = LP_TILE + 2 * M;
  for (int k = threadIdx.x; k < W; k += LP_THREADS) {
    const long long t = t0 - M + k;
    xs[k] = (t >= 0 && t < p.nt) ? __ldg(x + t) : 0.0f;
  }
  __syncthreads();

  // y[t] = sum_j h_j x[t - j]; with tl = t - t0 and k = j + M the sample
  // x[t - j] sits at xs[tl + 2M - k].
  float acc[LP_PER_THREAD];
#pragma unroll
  for (int q = 0; q < LP_PER_THREAD; ++q) acc[q] = 0.0f;
  for (int k = 0; k < ntap; ++k) {
    const float h = taps[k];
    const float* xk = xs + 2 * M - k + threadIdx.x;
#pragma unroll
    for (int q = 0; q < LP_PER_THREAD; ++q) acc[q] = fmaf(h, xk[q * LP_THREADS], acc[q]);
  }
  float* y = p.out + out_row * p.nt;
#pragma unroll
  for (int q = 0; q < LP_PER_THREAD; ++q) {
    const long long t = t0 + threadIdx.x + q * LP_THREADS;
    if (t < p.nt) y[t] = acc[q];
  }
}

__device__ __forceinline__ float vp_slope(const float* vp, const float* g, const float* mask,
                                          long long i) {
  const float v = vp[i];
  float d = -2.0f * g[i] / (v * v * v);
  if (mask) d *= mask[i];
  return d;
}

constexpr int UP_THREADS = 256;

__global__ void __launch_bounds__(UP_THREADS) k_vp_absmax(const float* __restrict__ vp,
                                                          const float* __restrict__ g,
                                                          const float* __restrict__ mask,
                                                          long long n, unsigned* __restrict__ out) {
  unsigned m = 0u;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(fabsf(vp_slope(vp, g, mask, i))));
  m = __reduce_max_sync(0xffffffffu, m);
  __shared__ unsigned wm[UP_THREADS / 32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned v = threadIdx.x < UP_THREADS / 32 ? wm[threadIdx.x] : 0u;
    v = __reduce_max_sync(0xffffffffu, v);
    if (threadIdx.x == 0 && v) atomicMax(out, v);
  }
}

__global__ void __launch_bounds__(UP_THREADS) k_vp_update(float* __restrict__ vp,
                                                          const float* __restrict__ g,
                                                          const float* __restrict__ mask,
                                                          long long n, const unsigned* __restrict__ smax,
                                                          float step, float vmin, float vmax) {
  const float s = __uint_as_float(*smax);
  const bool finite = s <= 3.4028234663852886e38f;   // false for Inf and NaN
  if (finite && s == 0.0f) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (!finite) {
      vp[i] = __uint_as_float(0x7fc00000u);
      continue;
    }
    const float d = vp_slope(vp, g, mask, i);
    const float v = vp[i] - step * (d / s);
    vp[i] = fminf(fmaxf(v, vmin), vmax);
  }
}

int grid_for(long long n, int threads) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  const long long need = (n + threads - 1) / threads;
  const long long cap = (long long)sms * 8;
  return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

fwi_status err(fwi_status s, const std::string& msg) {
  fwi::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" fwi_status fwi_lowpass(const float* in, int n_in, int rows, int nt, const int* ids,
                                  int n_ids, double dt, double f_max, int half_width, float* out,
                                  void* stream) {
  if (n_ids < 0 || n_in < 0 || rows < 0 || nt < 0)
    return err(FWI_ERR_INVALID_ARG, "fwi_lowpass: negative size");
  if (n_ids == 0 || rows == 0 || nt == 0) return FWI_OK;
  if (!in || !out || !ids) return err(FWI_ERR_INVALID_ARG, "fwi_lowpass: NULL array");
  if (rows > 65535) return err(FWI_ERR_INVALID_ARG, "fwi_lowpass: rows must be <= 65535");
  if (half_width < 0 || half_width > FWI_LOWPASS_MAX_HALF_WIDTH)
    return err(FWI_ERR_INVALID_ARG, "fwi_lowpass: half_width out of [0, FWI_LOWPASS_MAX_HALF_WIDTH]");
  if (!(dt > 0.0) || !std::isfinite(dt) || !(f_max > 0.0) || !std::isfinite(f_max))
    return err(FWI_ERR_INVALID_ARG, "fwi_lowpass: dt and f_max must be positive");
  for (int i = 0; i < n_ids; ++i)
    if (ids[i] < 0 || ids[i] >= n_in)
      return err(FWI_ERR_INVALID_ARG, "fwi_lowpass: id " + std::to_string(ids[i]) + " outside [0, n_in)");
  const long long in_elems = (long long)n_in * rows * nt;
  const long long out_elems = (long long)n_ids * rows * nt;
  if (in < out + out_elems && out < in + in_elems)
    return err(FWI_ERR_INVALID_ARG, "fwi_lowpass: out overlaps in");

  LowpassArgs p{};
  p.in = in;
  p.nt = nt;
  p.rows = rows;
  p.M = half_width;
  const double a = 2.0 * f_max * dt;
  p.a = (float)a;
  p.inv_m1 = (float)(1.0 / (half_width + 1.0));
  double norm = 0.0;
  for (int j = -half_width; j <= half_width; ++j) {
    const double x = kPi * a * j;
    const double s = j == 0 ? 1.0 : std::sin(x) / x;
    norm += s * 0.5 * (1.0 + std::cos(kPi * j / (half_width + 1.0)));
  }
  if (!(std::fabs(norm) > 1e-30)) return err(FWI_ERR_INVALID_ARG, "fwi_lowpass: degenerate taps");
  p.inv_norm = (float)(1.0 / norm);
  const size_t smem = sizeof(float) * (size_t)(2 * half_width + 1 + LP_TILE + 2 * half_width);
  const long long nseg = ((long long)nt + LP_TILE - 1) / LP_TILE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int c0 = 0; c0 < n_ids; c0 += LP_MAX_IDS) {
    const int nc = n_ids - c0 < LP_MAX_IDS ? n_ids - c0 : LP_MAX_IDS;
    for (int i = 0; i < nc; ++i) p.ids[i] = ids[c0 + i];
    p.out = out + (long long)c0 * rows * nt;
    k_lowpass<<<dim3((unsigned)nseg, (unsigned)rows, (unsigned)nc), LP_THREADS, smem, st>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return err(FWI_ERR_CUDA, std::string("fwi_lowpass: ") + cudaGetErrorString(e));
  }
  return FWI_OK;
}

extern "C" fwi_status fwi_vp_update(float* vp, const float* grad_m, const float* mask,
                                    long long n, float step, float vp_min, float vp_max,
                                    float* work, void* stream) {
  if (n < 0) return err(FWI_ERR_INVALID_ARG, "fwi_vp_update: negative size");
  if (n == 0) return FWI_OK;
  if (!vp || !grad_m || !work) return err(FWI_ERR_INVALID_ARG, "fwi_vp_update: NULL array");
  if (!(step >= 0.0f) || !std::isfinite(step) || !(vp_min <= vp_max) || !std::isfinite(vp_min) ||
      !std::isfinite(vp_max))
    return err(FWI_ERR_INVALID_ARG, "fwi_vp_update: need step >= 0 and finite vp_min <= vp_max");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned* smax = reinterpret_cast<unsigned*>(work);
  cudaError_t e = cudaMemsetAsync(smax, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return err(FWI_ERR_CUDA, std::string("fwi_vp_update: ") + cudaGetErrorString(e));
  const int grid = grid_for(n, UP_THREADS);
  k_vp_absmax<<<grid, UP_THREADS, 0, st>>>(vp, grad_m, mask, n, smax);
  k_vp_update<<<grid, UP_THREADS, 0, st>>>(vp, grad_m, mask, n, smax, step, vp_min, vp_max);
  e = cudaGetLastError();
  if (e != cudaSuccess) return err(FWI_ERR_CUDA, std::string("fwi_vp_update: ") + cudaGetErrorString(e));
  return FWI_OK;
}
