// Auxiliary kernels: model preparation, density gradient, receiver sampling,
// L2 misfit with residual (Sec. 3.2, `L2DistanceLoss`), trace transposition,
// final imaging term and gradient reduction over shot slots.
//
// All reductions run in a fixed order (block partials indexed by block, one
// final block) so repeated calls give bitwise-identical results.
#include "fwi_internal.cuh"

#include <math.h>

namespace fwi {

namespace {

// stats[0] = max vp bits, stats[1] = min vp bits, stats[2] = bad-value count
// vp holds the sound speed (param 0) or the squared slowness m = 1/vp^2 (param 1).
__global__ void k_model_prep(Layout L, const float* __restrict__ vp, const float* __restrict__ rho,
                             double dt, int param, float* __restrict__ kf, float* __restrict__ lnr,
                             unsigned int* __restrict__ stats) {
  const long long N = (long long)L.nx * L.ny * L.nz;
  unsigned int vmax = 0u, vmin = 0x7f800000u, bad = 0u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.nx);
    const long long t = i / L.nx;
    const int y = (int)(t % L.ny);
    const int z = (int)(t / L.ny);
    const long long pi = L.index(z, y, x);
    const float in = vp[i];
    if (!(in > 0.f) || !isfinite(in)) {
      ++bad;
      kf[pi] = 0.f;
    } else {
      // k = (vp dt)^2 = dt^2 / m
      const double k = param ? dt * dt / (double)in : ((double)in * dt) * ((double)in * dt);
      kf[pi] = (float)k;
      const float c = param ? (float)(1.0 / sqrt((double)in)) : in;
      const unsigned int bits = __float_as_uint(c);
      vmax = max(vmax, bits);
      vmin = min(vmin, bits);
    }
    if (rho) {
      const float r = rho[i];
      if (!(r > 0.f) || !isfinite(r)) {
        ++bad;
        lnr[pi] = 0.f;
      } else {
        lnr[pi] = (float)log((double)r);
      }
    }
  }
  // positive finite floats order like their bit patterns
  for (int o = 16; o > 0; o >>= 1) {
    vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(stats + 0, vmax);
    atomicMin(stats + 1, vmin);
    if (bad) atomicAdd(stats + 2, bad);
  }
}

// b_d = D1_d ln(rho) with ln(rho) replicated beyond the edges.
__global__ void k_density_grad(Layout L, const float* __restrict__ lnr, AxisW wx, AxisW wy,
                               AxisW wz, float* __restrict__ bx, float* __restrict__ by,
                               float* __restrict__ bz) {
  const long long N = (long long)L.nx * L.ny * L.nz;
  const int R = L.R;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.nx);
    const long long t = i / L.nx;
    const int y = (int)(t % L.ny);
    const int z = (int)(t / L.ny);
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int j = 1; j <= R; ++j) {
      const int xp = min(x + j, L.nx - 1), xm = max(x - j, 0);
      gx += (double)wx.w1[j] * ((double)lnr[L.index(z, y, xp)] - (double)lnr[L.index(z, y, xm)]);
      const int yp = min(y + j, L.ny - 1), ym = max(y - j, 0);
      gy += (double)wy.w1[j] * ((double)lnr[L.index(z, yp, x)] - (double)lnr[L.index(z, ym, x)]);
      if (L.ndim == 3) {
        const int zp = min(z + j, L.nz - 1), zm = max(z - j, 0);
        gz += (double)wz.w1[j] * ((double)lnr[L.index(zp, y, x)] - (double)lnr[L.index(zm, y, x)]);
      }
    }
    const long long pi = L.index(z, y, x);
    bx[pi] = (float)gx;
    by[pi] = (float)gy;
    if (bz) bz[pi] = (float)gz;
  }
}

__global__ void k_sample(StepParams p) {
  sample_receivers(p, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

__global__ void k_sample_slots(const float* __restrict__ u, long long fstride,
                               const int* __restrict__ node, const float* __restrict__ w, int nc,
                               int npts, int per_slot, float* __restrict__ out, long long off) {
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt < npts) {
    const float* ub = u + (long long)(pt / per_slot) * fstride;
    float acc = 0.f;
    for (int c = 0; c < nc; ++c) acc = fmaf(w[pt * nc + c], ub[node[pt * nc + c]], acc);
    out[off + pt] = acc;
  }
}

// Residual r = d - d_obs in place over the trace workspace [nt][B][nrec],
// traces copied out to [shot][nrec][nt], J partials per block (FP64).
// Block (32, 8) handles a 32 (time) x 32 (receiver) tile of one shot.
__global__ void k_misfit(const float* d_in, float* d_ws,
                         const float* __restrict__ obs, float* __restrict__ traces_out, int B,
                         int shot0, int nrec, int nt, double* __restrict__ partials,
                         int* __restrict__ nonfinite) {
  __shared__ float tobs[32][33];
  __shared__ float tout[32][33];
  __shared__ double red[256];
  const int n0 = blockIdx.x * 32, r0 = blockIdx.y * 32, b = blockIdx.z;
  const int s = shot0 + b;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (obs) {
    for (int rr = ty; rr < 32; rr += 8) {
      const int r = r0 + rr, n = n0 + tx;
      tobs[rr][tx] = (r < nrec && n < nt) ? obs[((long long)s * nrec + r) * nt + n] : 0.f;
    }
  }
  __syncthreads();
  double J = 0.0;
  bool bad = false;
  for (int nn = ty; nn < 32; nn += 8) {
    const int n = n0 + nn, r = r0 + tx;
    if (n < nt && r < nrec) {
      const long long o = ((long long)n * B + b) * nrec + r;
      const float d = d_in[o];
      if (!isfinite(d)) bad = true;
      if (obs) {
        const float res = d - tobs[tx][nn];
        d_ws[o] = res;
        J += 0.5 * (double)res * (double)res;
      }
      tout[tx][nn] = d;
    }
  }
  if (bad) atomicOr(nonfinite, 1);
  const int tid = ty * 32 + tx;
  red[tid] = J;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0 && partials) {
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partials[blk] = red[0];
  }
  if (traces_out) {
    for (int rr = ty; rr < 32; rr += 8) {
      const int r = r0 + rr, n = n0 + tx;
      if (r < nrec && n < nt) traces_out[((long long)s * nrec + r) * nt + n] = tout[rr][tx];
    }
  }
}

__global__ void k_sum_partials(const double* __restrict__ partials, int n, double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_image_only(const float4* __restrict__ lam, const float4* __restrict__ hist,
                             float4* __restrict__ g, long long f4, int nb, int S) {
  // f4: float4 per field; slots in fixed order so the sum is deterministic
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < f4;
       i += (long long)gridDim.x * blockDim.x) {
    for (int b = 0; b < nb; ++b) {
      const float4 l = lam[b * f4 + i], h = hist[b * f4 + i];
      float4* gp = g + (long long)(b / S) * f4 + i;
      float4 v = *gp;
      v.x = fmaf(-l.x, h.x, v.x);
      v.y = fmaf(-l.y, h.y, v.y);
      v.z = fmaf(-l.z, h.z, v.z);
      v.w = fmaf(-l.w, h.w, v.w);
      *gp = v;
    }
  }
}

__global__ void k_grad_finalize(Layout L, const float* __restrict__ g, int B, double inv_dt2,
                                float* __restrict__ out, int* __restrict__ nonfinite) {
  const long long N = (long long)L.nx * L.ny * L.nz;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.nx);
    const long long t = i / L.nx;
    const int y = (int)(t % L.ny);
    const int z = (int)(t / L.ny);
    const long long pi = L.index(z, y, x);
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += g[(long long)b * L.fstride + pi];
    const float v = (float)((double)s * inv_dt2);
    if (!isfinite(v)) bad = true;
    out[i] = v;
  }
  if (bad) atomicOr(nonfinite, 1);
}

int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_model_prep(const Layout& L, const float* vp, const float* rho, double dt,
                              int param, float* kf, float* lnr, unsigned int* stats,
                              cudaStream_t st) {
  const long long N = (long long)L.nx * L.ny * L.nz;
  k_model_prep<<<grid_for(N, 256), 256, 0, st>>>(L, vp, rho, dt, param, kf, lnr, stats);
  return cudaGetLastError();
}

cudaError_t launch_density_grad(const Layout& L, const float* lnr, const AxisW& wx,
                                const AxisW& wy, const AxisW& wz, float* bx, float* by,
                                float* bz, cudaStream_t st) {
  const long long N = (long long)L.nx * L.ny * L.nz;
  k_density_grad<<<grid_for(N, 256), 256, 0, st>>>(L, lnr, wx, wy, wz, bx, by, bz);
  return cudaGetLastError();
}

cudaError_t launch_sample(const StepParams& p, cudaStream_t st) {
  const long long n = (long long)p.B * p.nrec * (p.smp_group > 1 ? p.smp_group : 1);
  if (n == 0) return cudaSuccess;
  k_sample<<<(int)((n + 255) / 256), 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_sample_slots(const float* u, long long fstride, const int* node, const float* w,
                                int nc, int npts, int per_slot, float* out, long long off,
                                cudaStream_t st) {
  if (npts <= 0) return cudaSuccess;
  k_sample_slots<<<(npts + 127) / 128, 128, 0, st>>>(u, fstride, node, w, nc, npts, per_slot, out,
                                                     off);
  return cudaGetLastError();
}

int misfit_blocks(int nshots_batch, int nrec, int nt) {
  return ((nt + 31) / 32) * ((nrec + 31) / 32) * nshots_batch;
}

cudaError_t launch_misfit(const float* d_ws, const float* obs, float* traces_out, int B,
                          int shot0, int nshots_batch, int nrec, int nt, double* partials,
                          int* nonfinite, int npartials, cudaStream_t st) {
  dim3 grid((nt + 31) / 32, (nrec + 31) / 32, nshots_batch);
  k_misfit<<<grid, dim3(32, 8), 0, st>>>(d_ws, const_cast<float*>(d_ws), obs, traces_out, B,
                                         shot0, nrec, nt, partials, nonfinite);
  (void)npartials;
  return cudaGetLastError();
}

cudaError_t launch_traces_out(const float* d_ws, float* traces_out, int B, int shot0,
                              int nshots_batch, int nrec, int nt, int* nonfinite,
                              cudaStream_t st) {
  dim3 grid((nt + 31) / 32, (nrec + 31) / 32, nshots_batch);
  k_misfit<<<grid, dim3(32, 8), 0, st>>>(d_ws, nullptr, nullptr, traces_out, B, shot0, nrec, nt,
                                         nullptr, nonfinite);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* partials, int n, double* out, cudaStream_t st) {
  k_sum_partials<<<1, 256, 0, st>>>(partials, n, out);
  return cudaGetLastError();
}

cudaError_t launch_image_only(const Layout& L, const float* lam, const float* hist, float* g,
                              int nb, int S, cudaStream_t st) {
  const long long f4 = L.fstride / 4;
  k_image_only<<<grid_for(f4, 256), 256, 0, st>>>(reinterpret_cast<const float4*>(lam),
                                                  reinterpret_cast<const float4*>(hist),
                                                  reinterpret_cast<float4*>(g), f4, nb, S);
  return cudaGetLastError();
}

cudaError_t launch_grad_finalize(const Layout& L, const float* g, int B, double inv_dt2,
                                 float* grad_out, int* nonfinite, cudaStream_t st) {
  const long long N = (long long)L.nx * L.ny * L.nz;
  k_grad_finalize<<<grid_for(N, 256), 256, 0, st>>>(L, g, B, inv_dt2, grad_out, nonfinite);
  return cudaGetLastError();
}

}  // namespace fwi
