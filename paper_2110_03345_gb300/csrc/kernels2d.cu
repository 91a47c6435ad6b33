// 2D leapfrog step kernels (forward and adjoint) for sm_103a.
//
// One launch advances every shot slot of a batch by one time step of the
// damped leapfrog scheme for Eq. 10 (Sec. 2.4, no attenuation):
//   forward:  u^{n+1} = [2u^n - (1-a) u^{n-1} + k (L_rho u^n + s^n)] / (1+a)
//   adjoint:  l^{k-1} = [2l^k - (1-a) l^{k+1} + k (L_rho^T l^k + P^T r^k)] / (1+a)
// with k = (vp dt)^2, a = sigma dt / 2, L_rho = lap - grad(ln rho).grad and
// L_rho^T = lap + div(grad(ln rho) .) (central 8th/10th-order stencils).
// The adjoint step also applies the imaging condition of Sec. 2.2 (Eq. 8),
// g -= l^k * h^k with h^k = k (L u^k + s^k) stored by the forward pass, so
// the gradient with respect to m = 1/vp^2 is g / dt^2.
//
// Work decomposition: a CTA of 32 x BY threads owns a 128 x (RY*BY) tile
// of one shot; thread (tx, ty) computes a float4 of 4 consecutive x points in
// RY consecutive rows.  The tile plus its halo (radius R in y, 4 or 8 floats
// in x to keep float4 alignment) is staged once in shared memory with
// coalesced 16-byte loads; x derivatives read three (R=4) or five (R=5)
// float4 per row, y derivatives one float4 per row offset.  Sources (and, in
// the adjoint, receiver residuals) are added in the epilogue by the thread
// that owns the node, from a per-tile bucket list, so no atomics are used and
// results do not depend on scheduling.  The forward kernel's first threads
// also sample the receivers of u^n, which no thread writes during the step.
#include "fwi_internal.cuh"

namespace fwi {

namespace {

__device__ __forceinline__ float4 ldg4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st4(float* p, const float4& v) {
  *reinterpret_cast<float4*>(p) = v;
}
__device__ __forceinline__ float4 mul4(const float4& a, const float4& b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float get(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
__device__ __forceinline__ void unpack(const float4& t, float* v) {
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}


// One tile (bxi, byi) of shot slot b: the body shared by the single-problem
// kernel (indices from the launch grid) and the multi-problem kernel (indices
// from a unit table).  samp_rank is the CTA's rank among the CTAs of its
// problem, gx the problem's tile count along x.
template <int R, bool VD, bool ADJ, int RY, int BY>
__device__ __forceinline__ void step2d_tile(const StepParams& p, int bxi, int byi, int gx, int b,
                                            long long samp_rank, float4* smem) {
  constexpr int TX = TILE_X;
  constexpr int TY = RY * BY;
  constexpr int XH = (R <= 4) ? 4 : 8;   // x halo in floats (float4 aligned)
  constexpr int NL = XH / 4;             // halo float4 per side
  constexpr int SW = TX / 4 + 2 * NL;    // shared row width in float4
  constexpr int SH = TY + 2 * R;         // shared rows
  constexpr int NT = 32 * BY;
  constexpr int NV = 4 + 8 * NL;         // floats in one thread's x window
  constexpr int QW = TX / 4;             // psi_y row width in float4

  float4* s_u = smem;                    // [SH][SW]
  float4* s_px = s_u + SH * SW;          // adjoint, variable density: [TY][SW]
  float4* s_py = s_px + TY * SW;         // adjoint, variable density: [SH][QW]

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int x0 = bxi * TX, y0 = byi * TY;
  const long long fo = (long long)b * p.fstride;
  const float* __restrict__ u = p.u + fo;

  if (!ADJ && p.nrec > 0) sample_receivers(p, samp_rank * NT + tid);

  // Stage the tile and its halo.
  const long long base = (long long)(y0 + p.oy - R) * p.sx + (x0 + p.ox - XH);
  for (int i = tid; i < SH * SW; i += NT) {
    const int r = i / SW, c = i - r * SW;
    s_u[i] = ldg4(u + base + (long long)r * p.sx + 4 * c);
  }
  if (VD && ADJ) {
    // psi_x = b_x * lambda on the tile rows with the x halo,
    // psi_y = b_y * lambda on the tile columns with the y halo.
    for (int i = tid; i < TY * SW; i += NT) {
      const int r = i / SW, c = i - r * SW;
      const long long off = base + (long long)(r + R) * p.sx + 4 * c;
      s_px[i] = mul4(ldg4(p.bx + off), ldg4(u + off));
    }
    for (int i = tid; i < SH * QW; i += NT) {
      const int r = i / QW, c = i - r * QW;
      const long long off = base + (long long)r * p.sx + 4 * (c + NL);
      s_py[i] = mul4(ldg4(p.by + off), ldg4(u + off));
    }
  }
  __syncthreads();

  const int xg = x0 + 4 * tx;
  const float4 ax4 = ldg4(p.spx + xg);
  int e0 = 0, e1 = 0;
  if (p.inj_off) {
    const int t = b * p.ntiles + byi * gx + bxi;
    e0 = p.inj_off[t];
    e1 = p.inj_off[t + 1];
  }

#pragma unroll
  for (int iy = 0; iy < RY; ++iy) {
    const int ly = ty * RY + iy;
    const int yg = y0 + ly;
    const int srow = ly + R;

    float v[NV];
#pragma unroll
    for (int k = 0; k <= 2 * NL; ++k) unpack(s_u[srow * SW + tx + k], v + 4 * k);

    float acc[4];
    float d1x[4], d1y[4];
    // Second derivatives in the zero-sum form sum_j w_j (u_{+j} + u_{-j} - 2 u_0):
    // a constant field gives exactly 0 whatever the rounding of the FP32
    // weights (with w_0 written out, the rounded weights leave a residual of
    // ~1e-7 w_0 that acts as a spurious reaction term and shifts the phase
    // coherently over thousands of steps).
    float c2[4];
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) {
      const int c = 4 * NL + ix;
      c2[ix] = v[c] + v[c];
      float s = 0.f;
#pragma unroll
      for (int j = 1; j <= R; ++j) s = fmaf(p.wx.w2[j], (v[c + j] + v[c - j]) - c2[ix], s);
      acc[ix] = s;
      if (VD && !ADJ) {
        float d = 0.f;
#pragma unroll
        for (int j = 1; j <= R; ++j) d = fmaf(p.wx.w1[j], v[c + j] - v[c - j], d);
        d1x[ix] = d;
        d1y[ix] = 0.f;
      }
    }
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      const float4 a = s_u[(srow - j) * SW + tx + NL];
      const float4 c = s_u[(srow + j) * SW + tx + NL];
      acc[0] = fmaf(p.wy.w2[j], (a.x + c.x) - c2[0], acc[0]);
      acc[1] = fmaf(p.wy.w2[j], (a.y + c.y) - c2[1], acc[1]);
      acc[2] = fmaf(p.wy.w2[j], (a.z + c.z) - c2[2], acc[2]);
      acc[3] = fmaf(p.wy.w2[j], (a.w + c.w) - c2[3], acc[3]);
      if (VD && !ADJ) {
        d1y[0] = fmaf(p.wy.w1[j], c.x - a.x, d1y[0]);
        d1y[1] = fmaf(p.wy.w1[j], c.y - a.y, d1y[1]);
        d1y[2] = fmaf(p.wy.w1[j], c.z - a.z, d1y[2]);
        d1y[3] = fmaf(p.wy.w1[j], c.w - a.w, d1y[3]);
      }
    }

    const long long pi = (long long)(yg + p.oy) * p.sx + (xg + p.ox);
    if (VD && !ADJ) {
      // L_rho u = lap u - b . grad u
      const float4 bxv = ldg4(p.bx + pi), byv = ldg4(p.by + pi);
#pragma unroll
      for (int ix = 0; ix < 4; ++ix)
        acc[ix] -= get(bxv, ix) * d1x[ix] + get(byv, ix) * d1y[ix];
    }
    if (VD && ADJ) {
      // L_rho^T l = lap l + D1x(b_x l) + D1y(b_y l)
      float pv[NV];
#pragma unroll
      for (int k = 0; k <= 2 * NL; ++k) unpack(s_px[ly * SW + tx + k], pv + 4 * k);
#pragma unroll
      for (int ix = 0; ix < 4; ++ix) {
        const int c = 4 * NL + ix;
        float d = 0.f;
#pragma unroll
        for (int j = 1; j <= R; ++j) d = fmaf(p.wx.w1[j], pv[c + j] - pv[c - j], d);
        acc[ix] += d;
      }
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        const float4 a = s_py[(srow - j) * QW + tx];
        const float4 c = s_py[(srow + j) * QW + tx];
        acc[0] = fmaf(p.wy.w1[j], c.x - a.x, acc[0]);
        acc[1] = fmaf(p.wy.w1[j], c.y - a.y, acc[1]);
        acc[2] = fmaf(p.wy.w1[j], c.z - a.z, acc[2]);
        acc[3] = fmaf(p.wy.w1[j], c.w - a.w, acc[3]);
      }
    }

    // Point sources (forward) or receiver residuals (adjoint) owned by this thread.
    if (e1 > e0) {
      // only this row's entries (the bucket's per-row ranges)
      const int* rr = p.inj_row + (size_t)(b * p.ntiles + byi * gx + bxi) * (TY + 1);
      const int r1 = rr[ly + 1];
      for (int e = rr[ly]; e < r1; ++e) {
        const int elx = p.inj_loc[e] - ly * TX;
        if ((elx >> 2) == tx) {
          const float val = p.inj_w[e] * p.vals[p.inj_vidx[e] + p.step_off];
          const int ix = elx & 3;
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] += (q == ix) ? val : 0.f;
        }
      }
    }

    const float4 kk = ldg4(p.kf + pi);
    float* upp = p.up + fo + pi;
    const float4 uo = ld4(upp);
    const float ay = p.spy[yg];
    float res[4], upd[4];
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) {
      const float a = get(ax4, ix) + ay;
      const float h = get(kk, ix) * acc[ix];
      const float cen = v[4 * NL + ix];
      const float r = (2.f * cen - (1.f - a) * get(uo, ix) + h) * __frcp_rn(1.f + a);
      const bool in = (yg < p.ny) && (xg + ix < p.nx);
      res[ix] = in ? r : 0.f;
      upd[ix] = in ? h : 0.f;
    }
    st4(upp, make_float4(res[0], res[1], res[2], res[3]));
    if (!ADJ) {
      if (p.hist)
        __stcs(reinterpret_cast<float4*>(p.hist + fo + pi),
               make_float4(upd[0], upd[1], upd[2], upd[3]));
    } else if (p.image) {
      const float4 h = __ldcs(reinterpret_cast<const float4*>(p.hist + fo + pi));
      float* gp = p.g + fo + pi;
      float4 gg = ld4(gp);
      gg.x = fmaf(-v[4 * NL + 0], h.x, gg.x);
      gg.y = fmaf(-v[4 * NL + 1], h.y, gg.y);
      gg.z = fmaf(-v[4 * NL + 2], h.z, gg.z);
      gg.w = fmaf(-v[4 * NL + 3], h.w, gg.w);
      st4(gp, gg);
    }
  }
}

template <int R, bool VD, bool ADJ, int RY, int BY>
__global__ void __launch_bounds__(32 * BY)
k_step2d(const StepParams p) {
  extern __shared__ float4 smem[];
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  step2d_tile<R, VD, ADJ, RY, BY>(p, blockIdx.x, blockIdx.y, gridDim.x, blockIdx.z, blk, smem);
}

// Multi-problem step: CTA i advances unit units[i] (problem, tile, shot slot)
// by one time step of that problem, described by descs[problem]; the step
// index n is global (every problem started at n = 0).  The descriptor is copied
// to shared memory and completed with the fields that depend on n.
template <int R, bool VD, int RY, int BY>
__global__ void __launch_bounds__(32 * BY)
k_step2d_multi(const MultiDesc* __restrict__ descs, const MultiUnit* __restrict__ units, int n) {
  extern __shared__ float4 smem[];
  __shared__ StepParams sp;
  const MultiUnit un = units[blockIdx.x];
  {
    const int* src = reinterpret_cast<const int*>(&descs[un.prob].p);
    int* dst = reinterpret_cast<int*>(&sp);
    for (int i = threadIdx.y * 32 + threadIdx.x; i < (int)(sizeof(StepParams) / 4); i += 32 * BY)
      dst[i] = src[i];
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const MultiDesc& d = descs[un.prob];
    sp.u = (n & 1) ? d.U1 : d.U0;
    sp.up = (n & 1) ? d.U0 : d.U1;
    sp.step_off = n;
    sp.smp_off = (long long)n * sp.B * sp.nrec;
  }
  __syncthreads();
  step2d_tile<R, VD, false, RY, BY>(sp, un.tx, un.ty, descs[un.prob].gx, un.slot, un.rank, smem);
}

template <int R, bool VD, bool ADJ, int RY, int BY>
constexpr size_t smem_bytes() {
  constexpr int TY = RY * BY;
  constexpr int NL = (R <= 4) ? 1 : 2;
  constexpr int SW = TILE_X / 4 + 2 * NL;
  constexpr int SH = TY + 2 * R;
  size_t n = (size_t)SH * SW;
  if (VD && ADJ) n += (size_t)TY * SW + (size_t)SH * (TILE_X / 4);
  return n * sizeof(float4);
}

template <int R, bool VD, bool ADJ, int RY, int BY>
cudaError_t launch_t(const StepParams& p, cudaStream_t st) {
  constexpr int TY = RY * BY;
  constexpr size_t smem = smem_bytes<R, VD, ADJ, RY, BY>();
  static bool attr_set = false;   // per instantiation; set once per process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_step2d<R, VD, ADJ, RY, BY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((p.nx + TILE_X - 1) / TILE_X, (p.ny + TY - 1) / TY, p.B);
  dim3 block(32, BY);
  k_step2d<R, VD, ADJ, RY, BY><<<grid, block, smem, st>>>(p);
  return cudaGetLastError();
}

template <int R, bool VD, bool ADJ>
cudaError_t launch_tile(const StepParams& p, int tile, cudaStream_t st) {
  switch (tile) {
    case 1: return launch_t<R, VD, ADJ, 2, 16>(p, st);
    case 2: return launch_t<R, VD, ADJ, 4, 4>(p, st);
    case 3: return launch_t<R, VD, ADJ, 2, 8>(p, st);
    default: return launch_t<R, VD, ADJ, 4, 8>(p, st);
  }
}

template <int R, bool VD, bool ADJ>
size_t smem_tile(int tile) {
  switch (tile) {
    case 1: return smem_bytes<R, VD, ADJ, 2, 16>();
    case 2: return smem_bytes<R, VD, ADJ, 4, 4>();
    case 3: return smem_bytes<R, VD, ADJ, 2, 8>();
    default: return smem_bytes<R, VD, ADJ, 4, 8>();
  }
}

template <int R, bool VD>
cudaError_t launch_multi_t(const MultiDesc* descs, const MultiUnit* units, int nunits, int n,
                           cudaStream_t st) {
  constexpr size_t smem = smem_bytes<R, VD, false, 4, 8>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_step2d_multi<R, VD, 4, 8>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (nunits <= 0) return cudaSuccess;
  k_step2d_multi<R, VD, 4, 8><<<nunits, dim3(32, 8), smem, st>>>(descs, units, n);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step2d_multi(const MultiDesc* descs, const MultiUnit* units, int nunits, int n,
                                int R, bool vd, cudaStream_t st) {
  if (R == 4) return vd ? launch_multi_t<4, true>(descs, units, nunits, n, st)
                        : launch_multi_t<4, false>(descs, units, nunits, n, st);
  return vd ? launch_multi_t<5, true>(descs, units, nunits, n, st)
            : launch_multi_t<5, false>(descs, units, nunits, n, st);
}

cudaError_t launch_step2d(const StepParams& p, int R, bool vd, bool adj, int tile,
                          cudaStream_t st) {
  if (R == 4) {
    if (vd) return adj ? launch_tile<4, true, true>(p, tile, st) : launch_tile<4, true, false>(p, tile, st);
    return adj ? launch_tile<4, false, true>(p, tile, st) : launch_tile<4, false, false>(p, tile, st);
  }
  if (vd) return adj ? launch_tile<5, true, true>(p, tile, st) : launch_tile<5, true, false>(p, tile, st);
  return adj ? launch_tile<5, false, true>(p, tile, st) : launch_tile<5, false, false>(p, tile, st);
}

size_t step2d_smem(int R, bool vd, bool adj, int tile) {
  if (R == 4) {
    if (vd) return adj ? smem_tile<4, true, true>(tile) : smem_tile<4, true, false>(tile);
    return adj ? smem_tile<4, false, true>(tile) : smem_tile<4, false, false>(tile);
  }
  if (vd) return adj ? smem_tile<5, true, true>(tile) : smem_tile<5, true, false>(tile);
  return adj ? smem_tile<5, false, true>(tile) : smem_tile<5, false, false>(tile);
}

}  // namespace fwi
