// Step kernels of the extended schemes of Sec. 2.4: the fourth-order-in-time
// scheme and the power-law attenuation term of Eq. 10 (y = 0 and y = 2),
// forward and exact discrete adjoint with the imaging condition of Sec. 2.2
// (Eq. 8) fused into the adjoint step.
//
// With k = (vp dt)^2, a = sigma dt / 2 (sponge) and L the solver's spatial
// operator (L_rho forward, L_rho^T adjoint):
//
//  * fourth order in time (modified-equation scheme, two stencil passes):
//      pass 1 (EXT_KW):  kw = k (L u^n + s^n)
//      pass 2 (EXT_T4):  F  = kw + k (L kw + s^{n+1} - 2 s^n + s^{n-1}) / 12,
//                        u^{n+1} = [2u^n - (1-a) u^{n-1} + F] / (1+a);
//    the forward stores F and kw; the adjoint runs the same two passes with
//    L^T (pass A: ky = k L^T lambda^k; pass B: F = ky + k (L^T ky + 12 P^T r) / 12)
//    and accumulates g -= lambda^k F^k + ky^k kw^k / 12.
//  * attenuation y = 0 (EXT_ATT0): a += alpha0 vp dt per point; the forward
//    stores h - (alpha0 vp dt / 2)(u^{n+1} - u^{n-1}), the factor of the
//    gradient through the damping.
//  * attenuation y = 2 (EXT_ATT2): E = L u^n + s^n + beta (lap u^n - lap u^{n-1}) / dt,
//    beta = 2 alpha0 vp, with lap u^{n-1} kept per point (q, updated in
//    place); the adjoint adds (lap(beta lambda^k / dt) - its previous value);
//    the forward stores k E + (beta k / (2 dt))(lap u^n - lap u^{n-1}).
//  In every mode the adjoint's imaging term is g -= lambda^k * hist^k (plus the
//  kw term above), so the gradient with respect to m = 1/vp^2 is g / dt^2.
//
// Organisation: one grid point per thread.  2D: a CTA of 32 x 16 threads
// stages its tile plus halo in shared memory.  3D: a CTA of 32 x 8 threads
// streams a column along z over a chunk of planes with the column's 2R+1
// values in a register queue and the x-y plane (with halo) staged in shared
// memory.  Sources and receiver residuals come from the per-tile bucket
// lists (no atomics); second derivatives use the zero-sum form
// sum_j w_j (x_{+j} + x_{-j} - 2 x_0).
#include "fwi_internal.cuh"

namespace fwi {

namespace {

__device__ __forceinline__ void ext_sample(const StepParams& p, long long gid) {
  if (p.nrec > 0 && gid < (long long)p.B * p.nrec) {
    const int bb = (int)(gid / p.nrec);
    const int r = (int)(gid - (long long)bb * p.nrec);
    const float* ub = p.u + (long long)bb * p.fstride;
    float acc = 0.f;
    for (int c = 0; c < p.ncorner; ++c)
      acc = fmaf(p.smp_w[r * p.ncorner + c], ub[p.smp_node[r * p.ncorner + c]], acc);
    p.smp_out[p.smp_off + (long long)bb * p.nrec + r] = acc;
  }
}

__device__ __forceinline__ float ext_inject(const StepParams& p, int tile, int loc, float acc) {
  if (p.inj_off) {
    const int e0 = p.inj_off[tile], e1 = p.inj_off[tile + 1];
    for (int e = e0; e < e1; ++e)
      if (p.inj_loc[e] == loc)
        acc = fmaf(p.inj_scale * p.inj_w[e], p.vals[p.inj_vidx[e] + p.step_off], acc);
  }
  return acc;
}

// Update of one point: cen = x at the point, acc = (L x + injection), lap =
// its plain Laplacian part, lc = lap(att x) (y = 2 adjoint), a0 = sponge.
template <bool ADJ, int MODE>
__device__ __forceinline__ void ext_update(const StepParams& p, long long fo, long long pi,
                                           float cen, float acc, float lap, float lc, float a0) {
  const float k = __ldg(p.kf + pi);
  float* upp = p.up + fo + pi;
  if (MODE == EXT_KW) {
    p.out[fo + pi] = k * acc;
  } else if (MODE == EXT_T4) {
    const float F = cen + __fdiv_rn(k * acc, 12.f);
    const float uc = p.u[fo + pi];
    const float uo = *upp;
    *upp = (2.f * uc - (1.f - a0) * uo + F) * __frcp_rn(1.f + a0);
    if (!ADJ) {
      if (p.hist) {
        p.hist[fo + pi] = F;
        p.hist2[fo + pi] = cen;
      }
    } else if (p.image) {
      float* gp = p.g + fo + pi;
      *gp = *gp - (uc * p.hist[fo + pi] + __fdiv_rn(cen * p.hist2[fo + pi], 12.f));
    }
  } else if (MODE == EXT_ATT0) {
    const float at = __ldg(p.att + pi);
    const float a = a0 + at;
    const float uo = *upp;
    const float h = k * acc;
    const float r = (2.f * cen - (1.f - a) * uo + h) * __frcp_rn(1.f + a);
    *upp = r;
    if (!ADJ) {
      if (p.hist) p.hist[fo + pi] = h - 0.5f * at * (r - uo);
    } else if (p.image) {
      float* gp = p.g + fo + pi;
      *gp = fmaf(-cen, p.hist[fo + pi], *gp);
    }
  } else {   // EXT_ATT2
    const float cf = __ldg(p.att + pi);
    float* qp = p.q + fo + pi;
    const float qo = *qp;
    float E, extra = 0.f;
    if (!ADJ) {
      const float dl = lap - qo;
      E = fmaf(cf, dl, acc);
      *qp = lap;
      extra = 0.5f * k * cf * dl;
    } else {
      E = acc + (lc - qo);
      *qp = lc;
    }
    const float h = k * E;
    const float uo = *upp;
    *upp = (2.f * cen - (1.f - a0) * uo + h) * __frcp_rn(1.f + a0);
    if (!ADJ) {
      if (p.hist) p.hist[fo + pi] = h + extra;
    } else if (p.image) {
      float* gp = p.g + fo + pi;
      *gp = fmaf(-cen, p.hist[fo + pi], *gp);
    }
  }
}

template <int R, bool VD, bool ADJ, int MODE>
__global__ void __launch_bounds__(EXT_TX * EXT_TY2) k_ext2d(const StepParams p) {
  constexpr int TX = EXT_TX, TY = EXT_TY2;
  constexpr int SW = TX + 2 * R, SH = TY + 2 * R;
  constexpr int NT = TX * TY;
  constexpr bool PSI = VD && ADJ;                    // b_d x for L^T
  constexpr bool CL = (MODE == EXT_ATT2) && ADJ;     // att x for lap(att x)
  __shared__ float s_x[SH][SW];
  __shared__ float s_px[PSI ? TY : 1][PSI ? SW : 1];
  __shared__ float s_py[PSI ? SH : 1][PSI ? TX : 1];
  __shared__ float s_c[CL ? SH : 1][CL ? SW : 1];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int b = blockIdx.z;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const long long fo = (long long)b * p.fstride;
  const float* __restrict__ X = p.x + fo;
  if (!ADJ) {
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    ext_sample(p, blk * NT + tid);
  }
  const long long base = (long long)(y0 + p.oy - R) * p.sx + (x0 + p.ox - R);
  for (int i = tid; i < SH * SW; i += NT) {
    const int r = i / SW, c = i - r * SW;
    const long long o = base + (long long)r * p.sx + c;
    const float v = X[o];
    s_x[r][c] = v;
    if (CL) s_c[r][c] = __ldg(p.att + o) * v;
  }
  if (PSI) {
    for (int i = tid; i < TY * SW; i += NT) {
      const int r = i / SW, c = i - r * SW;
      const long long o = base + (long long)(r + R) * p.sx + c;
      s_px[r][c] = __ldg(p.bx + o) * X[o];
    }
    for (int i = tid; i < SH * TX; i += NT) {
      const int r = i / TX, c = i - r * TX;
      const long long o = base + (long long)r * p.sx + c + R;
      s_py[r][c] = __ldg(p.by + o) * X[o];
    }
  }
  __syncthreads();

  const int xg = x0 + tx, yg = y0 + ty;
  const int cx = tx + R, cy = ty + R;
  const float cen = s_x[cy][cx];
  const float c2 = cen + cen;
  float lap = 0.f;
#pragma unroll
  for (int j = 1; j <= R; ++j) lap = fmaf(p.wx.w2[j], (s_x[cy][cx + j] + s_x[cy][cx - j]) - c2, lap);
#pragma unroll
  for (int j = 1; j <= R; ++j) lap = fmaf(p.wy.w2[j], (s_x[cy + j][cx] + s_x[cy - j][cx]) - c2, lap);
  float acc = lap;
  const long long pi = (long long)(yg + p.oy) * p.sx + (xg + p.ox);
  if (VD && !ADJ) {
    float dx = 0.f, dy = 0.f;
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      dx = fmaf(p.wx.w1[j], s_x[cy][cx + j] - s_x[cy][cx - j], dx);
      dy = fmaf(p.wy.w1[j], s_x[cy + j][cx] - s_x[cy - j][cx], dy);
    }
    acc -= __ldg(p.bx + pi) * dx + __ldg(p.by + pi) * dy;
  }
  if (PSI) {
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      acc = fmaf(p.wx.w1[j], s_px[ty][cx + j] - s_px[ty][cx - j], acc);
      acc = fmaf(p.wy.w1[j], s_py[cy + j][tx] - s_py[cy - j][tx], acc);
    }
  }
  float lc = 0.f;
  if (CL) {
    const float cc2 = 2.f * s_c[cy][cx];
#pragma unroll
    for (int j = 1; j <= R; ++j) lc = fmaf(p.wx.w2[j], (s_c[cy][cx + j] + s_c[cy][cx - j]) - cc2, lc);
#pragma unroll
    for (int j = 1; j <= R; ++j) lc = fmaf(p.wy.w2[j], (s_c[cy + j][cx] + s_c[cy - j][cx]) - cc2, lc);
  }
  acc = ext_inject(p, b * p.ntiles + blockIdx.y * gridDim.x + blockIdx.x, ty * TX + tx, acc);
  if (xg < p.nx && yg < p.ny)
    ext_update<ADJ, MODE>(p, fo, pi, cen, acc, lap, lc, p.spx[xg] + p.spy[yg]);
}

template <int R, bool VD, bool ADJ, int MODE>
__global__ void __launch_bounds__(EXT_TX * EXT_TY3) k_ext3d(const StepParams p) {
  constexpr int TX = EXT_TX, TY = EXT_TY3;
  constexpr int SW = TX + 2 * R, SH = TY + 2 * R;
  constexpr int NT = TX * TY;
  constexpr int Q = 2 * R + 1;
  constexpr bool PSI = VD && ADJ;
  constexpr bool CL = (MODE == EXT_ATT2) && ADJ;
  __shared__ float s_x[SH][SW];
  __shared__ float s_px[PSI ? TY : 1][PSI ? SW : 1];
  __shared__ float s_py[PSI ? SH : 1][PSI ? TX : 1];
  __shared__ float s_c[CL ? SH : 1][CL ? SW : 1];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int b = blockIdx.z / p.nzc;
  const int zc = blockIdx.z - b * p.nzc;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = zc * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.nz);
  const long long fo = (long long)b * p.fstride;
  const float* __restrict__ X = p.x + fo;
  const int xg = x0 + tx, yg = y0 + ty;
  const long long col = (long long)(yg + p.oy) * p.sx + (xg + p.ox);
  if (!ADJ) {
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    ext_sample(p, blk * NT + tid);
  }
  // register queues along z: q[j] = x at plane z - R + j of this column
  float q[Q];
  float qz[PSI ? Q : 1];
  float qc[CL ? Q : 1];
#pragma unroll
  for (int j = 0; j < Q - 1; ++j) {
    const long long o = col + (long long)(z0 - R + j + p.oz) * p.sxy;
    q[j] = X[o];
    if (PSI) qz[j] = __ldg(p.bz + o) * q[j];
    if (CL) qc[j] = __ldg(p.att + o) * q[j];
  }
  const float axy = p.spx[xg] + p.spy[yg];
  const bool in_xy = (xg < p.nx) && (yg < p.ny);
  const int tile = b * p.ntiles + (zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int cx = tx + R, cy = ty + R;

  for (int z = z0; z < z1; ++z) {
    const long long pz = (long long)(z + p.oz) * p.sxy;
    {
      const long long o = col + pz + (long long)R * p.sxy;
      q[Q - 1] = X[o];
      if (PSI) qz[Q - 1] = __ldg(p.bz + o) * q[Q - 1];
      if (CL) qc[Q - 1] = __ldg(p.att + o) * q[Q - 1];
    }
    __syncthreads();   // the previous plane's readers are done with the shared tiles
    const long long pb = pz + (long long)(y0 + p.oy - R) * p.sx + (x0 + p.ox - R);
    for (int i = tid; i < SH * SW; i += NT) {
      const int r = i / SW, c = i - r * SW;
      const long long o = pb + (long long)r * p.sx + c;
      const float v = X[o];
      s_x[r][c] = v;
      if (CL) s_c[r][c] = __ldg(p.att + o) * v;
    }
    if (PSI) {
      for (int i = tid; i < TY * SW; i += NT) {
        const int r = i / SW, c = i - r * SW;
        const long long o = pb + (long long)(r + R) * p.sx + c;
        s_px[r][c] = __ldg(p.bx + o) * X[o];
      }
      for (int i = tid; i < SH * TX; i += NT) {
        const int r = i / TX, c = i - r * TX;
        const long long o = pb + (long long)r * p.sx + c + R;
        s_py[r][c] = __ldg(p.by + o) * X[o];
      }
    }
    __syncthreads();

    const float cen = q[R];
    const float c2 = cen + cen;
    float lap = 0.f;
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      lap = fmaf(p.wx.w2[j], (s_x[cy][cx + j] + s_x[cy][cx - j]) - c2, lap);
      lap = fmaf(p.wy.w2[j], (s_x[cy + j][cx] + s_x[cy - j][cx]) - c2, lap);
      lap = fmaf(p.wz.w2[j], (q[R + j] + q[R - j]) - c2, lap);
    }
    float acc = lap;
    const long long idx = col + pz;
    if (VD && !ADJ) {
      float dx = 0.f, dy = 0.f, dz = 0.f;
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        dx = fmaf(p.wx.w1[j], s_x[cy][cx + j] - s_x[cy][cx - j], dx);
        dy = fmaf(p.wy.w1[j], s_x[cy + j][cx] - s_x[cy - j][cx], dy);
        dz = fmaf(p.wz.w1[j], q[R + j] - q[R - j], dz);
      }
      acc -= __ldg(p.bx + idx) * dx + __ldg(p.by + idx) * dy + __ldg(p.bz + idx) * dz;
    }
    if (PSI) {
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        acc = fmaf(p.wx.w1[j], s_px[ty][cx + j] - s_px[ty][cx - j], acc);
        acc = fmaf(p.wy.w1[j], s_py[cy + j][tx] - s_py[cy - j][tx], acc);
        acc = fmaf(p.wz.w1[j], qz[R + j] - qz[R - j], acc);
      }
    }
    float lc = 0.f;
    if (CL) {
      const float cc2 = 2.f * qc[R];
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        lc = fmaf(p.wx.w2[j], (s_c[cy][cx + j] + s_c[cy][cx - j]) - cc2, lc);
        lc = fmaf(p.wy.w2[j], (s_c[cy + j][cx] + s_c[cy - j][cx]) - cc2, lc);
        lc = fmaf(p.wz.w2[j], (qc[R + j] + qc[R - j]) - cc2, lc);
      }
    }
    acc = ext_inject(p, tile, ((z - z0) * TY + ty) * TX + tx, acc);
    if (in_xy) ext_update<ADJ, MODE>(p, fo, idx, cen, acc, lap, lc, axy + p.spz[z]);
#pragma unroll
    for (int j = 0; j < Q - 1; ++j) {
      q[j] = q[j + 1];
      if (PSI) qz[j] = qz[j + 1];
      if (CL) qc[j] = qc[j + 1];
    }
  }
}

template <int R, bool VD, bool ADJ, int MODE>
cudaError_t launch_m(const StepParams& p, int ndim, cudaStream_t st) {
  if (ndim == 2) {
    dim3 grid((p.nx + EXT_TX - 1) / EXT_TX, (p.ny + EXT_TY2 - 1) / EXT_TY2, p.B);
    k_ext2d<R, VD, ADJ, MODE><<<grid, dim3(EXT_TX, EXT_TY2), 0, st>>>(p);
  } else {
    dim3 grid((p.nx + EXT_TX - 1) / EXT_TX, (p.ny + EXT_TY3 - 1) / EXT_TY3, p.B * p.nzc);
    k_ext3d<R, VD, ADJ, MODE><<<grid, dim3(EXT_TX, EXT_TY3), 0, st>>>(p);
  }
  return cudaGetLastError();
}

template <int R, bool VD, bool ADJ>
cudaError_t launch_mode(const StepParams& p, int ndim, int mode, cudaStream_t st) {
  switch (mode) {
    case EXT_KW: return launch_m<R, VD, ADJ, EXT_KW>(p, ndim, st);
    case EXT_T4: return launch_m<R, VD, ADJ, EXT_T4>(p, ndim, st);
    case EXT_ATT0: return launch_m<R, VD, ADJ, EXT_ATT0>(p, ndim, st);
    default: return launch_m<R, VD, ADJ, EXT_ATT2>(p, ndim, st);
  }
}

__global__ void k_second_difference(const float* __restrict__ q, float* __restrict__ out,
                                    long long rows, int nt) {
  const long long n = rows * nt;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i % nt);
    const float c = q[i];
    const float a = t > 0 ? q[i - 1] : 0.f;
    const float b = t + 1 < nt ? q[i + 1] : 0.f;
    out[i] = (a + b) - 2.f * c;
  }
}

// stats[0] = largest coefficient (bits of a non-negative float), stats[1] =
// number of negative or non-finite alpha0 values (their coefficient is 0)
__global__ void k_att_prep(Layout L, const float* __restrict__ vp, int param,
                           const float* __restrict__ alpha0, int y, double dt,
                           float* __restrict__ att, unsigned int* __restrict__ stats) {
  const long long N = (long long)L.nx * L.ny * L.nz;
  unsigned int amax = 0u, bad = 0u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.nx);
    const long long t = i / L.nx;
    const int yy = (int)(t % L.ny);
    const int z = (int)(t / L.ny);
    const double v = param ? 1.0 / sqrt((double)vp[i]) : (double)vp[i];
    const float a = alpha0[i];
    float c = 0.f;
    if (!(a >= 0.f) || !isfinite(a)) ++bad;
    else c = (float)(y == 0 ? (double)a * v * dt : 2.0 * (double)a * v / dt);
    att[L.index(z, yy, x)] = c;
    amax = max(amax, __float_as_uint(c));
  }
  for (int o = 16; o > 0; o >>= 1) {
    amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(stats + 0, amax);
    if (bad) atomicAdd(stats + 1, bad);
  }
}

}  // namespace

cudaError_t launch_ext(const StepParams& p, int ndim, int R, bool vd, bool adj, int mode,
                       cudaStream_t st) {
  if (R == 4) {
    if (vd) return adj ? launch_mode<4, true, true>(p, ndim, mode, st) : launch_mode<4, true, false>(p, ndim, mode, st);
    return adj ? launch_mode<4, false, true>(p, ndim, mode, st) : launch_mode<4, false, false>(p, ndim, mode, st);
  }
  if (vd) return adj ? launch_mode<5, true, true>(p, ndim, mode, st) : launch_mode<5, true, false>(p, ndim, mode, st);
  return adj ? launch_mode<5, false, true>(p, ndim, mode, st) : launch_mode<5, false, false>(p, ndim, mode, st);
}

cudaError_t launch_second_difference(const float* q, float* out, long long rows, int nt,
                                     cudaStream_t st) {
  const long long n = rows * nt;
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  k_second_difference<<<(int)blocks, 256, 0, st>>>(q, out, rows, nt);
  return cudaGetLastError();
}

cudaError_t launch_att_prep(const Layout& L, const float* vp, int param, const float* alpha0,
                            int y, double dt, float* att, unsigned int* stats, cudaStream_t st) {
  const long long N = (long long)L.nx * L.ny * L.nz;
  long long blocks = (N + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  k_att_prep<<<(int)blocks, 256, 0, st>>>(L, vp, param, alpha0, y, dt, att, stats);
  return cudaGetLastError();
}

}  // namespace fwi

namespace fwi {

namespace {

// g[b] -= lam[b] F[b] + ky[b] kw[b] / 12 over the nb slots of a batch (the
// fourth-order imaging term of lambda^0, which no adjoint step follows).
__global__ void k_image_t4(const float* __restrict__ lam, const float* __restrict__ ky,
                           const float* __restrict__ F, const float* __restrict__ kw,
                           float* __restrict__ g, long long fs, int nb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < fs;
       i += (long long)gridDim.x * blockDim.x) {
    for (int b = 0; b < nb; ++b) {
      const long long o = (long long)b * fs + i;
      g[o] = g[o] - (lam[o] * F[o] + __fdiv_rn(ky[o] * kw[o], 12.f));
    }
  }
}

}  // namespace

cudaError_t launch_image_t4(const Layout& L, const float* lam, const float* ky, const float* F,
                            const float* kw, float* g, int nb, cudaStream_t st) {
  const long long fs = L.fstride;
  long long blocks = (fs + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  k_image_t4<<<(int)blocks, 256, 0, st>>>(lam, ky, F, kw, g, fs, nb);
  return cudaGetLastError();
}

}  // namespace fwi
