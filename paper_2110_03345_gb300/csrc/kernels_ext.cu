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
// Organisation.  2D (the steps themselves run on the TMA shot-loop kernels of
// kernels2d_tma_ext.cu; this one serves the adjoint's last k L^T lambda^0
// pass): a CTA of 32 x 16 threads stages a 128 x 16 tile plus halo in shared
// memory with 16-byte loads, each thread updating a float4 of x points.  3D: one grid point per thread, a CTA of 32 x 8 threads
// streams a column along z over a chunk of planes with the column's 2R+1
// values in a register queue and the x-y plane (with halo) staged in shared
// memory.  Sources and receiver residuals come from the per-tile bucket
// lists (no atomics); second derivatives use the zero-sum form
// sum_j w_j (x_{+j} + x_{-j} - 2 x_0).
#include "fwi_internal.cuh"

namespace fwi {

namespace {


constexpr float INV12 = 1.f / 12.f;   // the 1/12 of the fourth-order terms, rounded once

// Per-point operands of one plane of the 3D kernel, loaded at the top of the
// plane's trip so that their latency overlaps the plane staging, the barrier
// and the stencil (each point is read and written by its own thread only).
template <bool VD, bool ADJ, int MODE>
struct PointOps {
  float k, uo, uc, at, qo, h, h2, g, bx, by, bz;
  __device__ __forceinline__ void load(const StepParams& p, long long fo, long long pi) {
    k = __ldg(p.kf + pi);
    if (MODE != EXT_KW) uo = p.up[fo + pi];
    if (MODE == EXT_T4) uc = p.u[fo + pi];
    if (MODE == EXT_ATT0 || MODE == EXT_ATT2) at = __ldg(p.att + pi);
    if (MODE == EXT_ATT2) qo = p.q[fo + pi];
    if (ADJ && MODE != EXT_KW && p.image) {
      h = p.hist[fo + pi];
      if (MODE == EXT_T4) h2 = p.hist2[fo + pi];
      g = p.g[fo + pi];
    }
    if (VD && !ADJ) {
      bx = __ldg(p.bx + pi);
      by = __ldg(p.by + pi);
      bz = __ldg(p.bz + pi);
    }
  }
};

// Update of one point: cen = x at the point, acc = (L x + injection), lap =
// its plain Laplacian part, lc = lap(att x) (y = 2 adjoint), a0 = sponge,
// o = the point's operands.
template <bool VD, bool ADJ, int MODE>
__device__ __forceinline__ void ext_update(const StepParams& p, long long fo, long long pi,
                                           float cen, float acc, float lap, float lc, float a0,
                                           const PointOps<VD, ADJ, MODE>& o) {
  const float k = o.k;
  float* upp = p.up + fo + pi;
  if (MODE == EXT_KW) {
    p.out[fo + pi] = k * acc;
  } else if (MODE == EXT_T4) {
    const float F = fmaf(k * acc, INV12, cen);
    const float uc = o.uc;
    *upp = (2.f * uc - (1.f - a0) * o.uo + F) * __frcp_rn(1.f + a0);
    if (!ADJ) {
      if (p.hist) {
        p.hist[fo + pi] = F;
        p.hist2[fo + pi] = cen;
      }
    } else if (p.image) {
      p.g[fo + pi] = o.g - fmaf(cen * o.h2, INV12, uc * o.h);
    }
  } else if (MODE == EXT_ATT0) {
    const float at = o.at;
    const float a = a0 + at;
    const float uo = o.uo;
    const float h = k * acc;
    const float r = (2.f * cen - (1.f - a) * uo + h) * __frcp_rn(1.f + a);
    *upp = r;
    if (!ADJ) {
      if (p.hist) p.hist[fo + pi] = h - 0.5f * at * (r - uo);
    } else if (p.image) {
      p.g[fo + pi] = fmaf(-cen, o.h, o.g);
    }
  } else {   // EXT_ATT2
    const float cf = o.at;
    const float qo = o.qo;
    float E, extra = 0.f;
    float* qp = p.q + fo + pi;
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
    *upp = (2.f * cen - (1.f - a0) * o.uo + h) * __frcp_rn(1.f + a0);
    if (!ADJ) {
      if (p.hist) p.hist[fo + pi] = h + extra;
    } else if (p.image) {
      p.g[fo + pi] = fmaf(-cen, o.h, o.g);
    }
  }
}

__device__ __forceinline__ float4 ldg4(const float* q) {
  return __ldg(reinterpret_cast<const float4*>(q));
}
__device__ __forceinline__ float4 ld4(const float* q) { return *reinterpret_cast<const float4*>(q); }
__device__ __forceinline__ void st4(float* q, const float4& v) { *reinterpret_cast<float4*>(q) = v; }
__device__ __forceinline__ float4 mul4(const float4& a, const float4& b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ void unpack(const float4& t, float* v) {
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ float4 pack(const float* v) { return make_float4(v[0], v[1], v[2], v[3]); }

// Shared-memory layout of the 2D kernel (float4 units): the stencil input
// tile with halo [SH][SW]; for the variable-density adjoint b_x x on the tile
// rows [TY][SW] and b_y x on the tile columns [SH][QW]; for the y = 2
// adjoint att x in the same two shapes.
template <int R, bool VD, bool ADJ, int MODE>
struct Ext2 {
  static constexpr int TX = EXT_TX2, TY = EXT_TY2;
  static constexpr int XH = (R <= 4) ? 4 : 8, NL = XH / 4;
  static constexpr int SW = TX / 4 + 2 * NL, SH = TY + 2 * R, QW = TX / 4;
  static constexpr bool PSI = VD && ADJ;
  static constexpr bool CL = (MODE == EXT_ATT2) && ADJ;
  static constexpr int CROSS = TY * SW + SH * QW;
  static constexpr size_t SMEM = ((size_t)SH * SW + (PSI ? CROSS : 0) + (CL ? CROSS : 0)) * 16;
};

// One 128 x 16 tile of one shot; thread (tx, ty) owns the float4 of x points
// 4 tx .. 4 tx + 3 of row ty.
template <int R, bool VD, bool ADJ, int MODE>
__global__ void __launch_bounds__(EXT_TX2 / 4 * EXT_TY2) k_ext2d(const StepParams p) {
  using G = Ext2<R, VD, ADJ, MODE>;
  constexpr int TX = G::TX, TY = G::TY, NL = G::NL, SW = G::SW, SH = G::SH, QW = G::QW;
  constexpr int NT = TX / 4 * TY;
  constexpr int NV = 4 + 8 * NL;
  constexpr bool PSI = G::PSI, CL = G::CL;
  extern __shared__ __align__(16) float4 sm[];
  float4* s_x = sm;                          // [SH][SW]
  float4* s_px = s_x + SH * SW;              // PSI: b_x x [TY][SW], then b_y x [SH][QW]
  float4* s_py = s_px + TY * SW;
  float4* s_cx = s_x + SH * SW + (PSI ? G::CROSS : 0);   // CL: att x, same shapes
  float4* s_cy = s_cx + TY * SW;

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * (TX / 4) + tx;
  const int b = blockIdx.z;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const long long fo = (long long)b * p.fstride;
  const float* __restrict__ X = p.x + fo;
  if (!ADJ) {
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    sample_receivers(p, blk * NT + tid);
  }
  const long long base = (long long)(y0 + p.oy - R) * p.sx + (x0 + p.ox - G::XH);
  for (int i = tid; i < SH * SW; i += NT) {
    const int r = i / SW, c = i - r * SW;
    s_x[i] = ldg4(X + base + (long long)r * p.sx + 4 * c);
  }
  if (PSI || CL) {
    for (int i = tid; i < TY * SW; i += NT) {
      const int r = i / SW, c = i - r * SW;
      const long long o = base + (long long)(r + R) * p.sx + 4 * c;
      const float4 xv = ldg4(X + o);
      if (PSI) s_px[i] = mul4(ldg4(p.bx + o), xv);
      if (CL) s_cx[i] = mul4(ldg4(p.att + o), xv);
    }
    for (int i = tid; i < SH * QW; i += NT) {
      const int r = i / QW, c = i - r * QW;
      const long long o = base + (long long)r * p.sx + 4 * (c + NL);
      const float4 xv = ldg4(X + o);
      if (PSI) s_py[i] = mul4(ldg4(p.by + o), xv);
      if (CL) s_cy[i] = mul4(ldg4(p.att + o), xv);
    }
  }
  __syncthreads();

  const int ly = ty, yg = y0 + ly, srow = ly + R;
  const int xg = x0 + 4 * tx;
  float v[NV];
#pragma unroll
  for (int q = 0; q <= 2 * NL; ++q) unpack(s_x[srow * SW + tx + q], v + 4 * q);
  float acc[4], c2[4], cen[4];
#pragma unroll
  for (int ix = 0; ix < 4; ++ix) {
    const int c = 4 * NL + ix;
    cen[ix] = v[c];
    c2[ix] = v[c] + v[c];
    float t = 0.f;
#pragma unroll
    for (int j = 1; j <= R; ++j) t = fmaf(p.wx.w2[j], (v[c + j] + v[c - j]) - c2[ix], t);
    acc[ix] = t;
  }
  float d1y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    const float4 a = s_x[(srow - j) * SW + tx + NL];
    const float4 c = s_x[(srow + j) * SW + tx + NL];
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
  float lap[4];
#pragma unroll
  for (int ix = 0; ix < 4; ++ix) lap[ix] = acc[ix];
  const long long pi = (long long)(yg + p.oy) * p.sx + (xg + p.ox);
  if (VD && !ADJ) {   // L_rho u = lap u - b . grad u
    float bxv[4], byv[4];
    unpack(ldg4(p.bx + pi), bxv);
    unpack(ldg4(p.by + pi), byv);
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) {
      const int c = 4 * NL + ix;
      float d = 0.f;
#pragma unroll
      for (int j = 1; j <= R; ++j) d = fmaf(p.wx.w1[j], v[c + j] - v[c - j], d);
      acc[ix] -= bxv[ix] * d + byv[ix] * d1y[ix];
    }
  }
  if (PSI) {          // L_rho^T x = lap x + D1x(b_x x) + D1y(b_y x)
    float pv[NV];
#pragma unroll
    for (int q = 0; q <= 2 * NL; ++q) unpack(s_px[ly * SW + tx + q], pv + 4 * q);
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) {
      const int c = 4 * NL + ix;
#pragma unroll
      for (int j = 1; j <= R; ++j) acc[ix] = fmaf(p.wx.w1[j], pv[c + j] - pv[c - j], acc[ix]);
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
  float lc[4] = {0.f, 0.f, 0.f, 0.f};
  if (CL) {           // lap(att x)
    float cv[NV];
#pragma unroll
    for (int q = 0; q <= 2 * NL; ++q) unpack(s_cx[ly * SW + tx + q], cv + 4 * q);
    float cc2[4];
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) {
      const int c = 4 * NL + ix;
      cc2[ix] = 2.f * cv[c];
#pragma unroll
      for (int j = 1; j <= R; ++j) lc[ix] = fmaf(p.wx.w2[j], (cv[c + j] + cv[c - j]) - cc2[ix], lc[ix]);
    }
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      const float4 a = s_cy[(srow - j) * QW + tx];
      const float4 c = s_cy[(srow + j) * QW + tx];
      lc[0] = fmaf(p.wy.w2[j], (a.x + c.x) - cc2[0], lc[0]);
      lc[1] = fmaf(p.wy.w2[j], (a.y + c.y) - cc2[1], lc[1]);
      lc[2] = fmaf(p.wy.w2[j], (a.z + c.z) - cc2[2], lc[2]);
      lc[3] = fmaf(p.wy.w2[j], (a.w + c.w) - cc2[3], lc[3]);
    }
  }
  if (p.inj_off) {    // this row's entries of the tile's bucket
    const int t = b * p.ntiles + blockIdx.y * gridDim.x + blockIdx.x;
    if (p.inj_off[t + 1] > p.inj_off[t]) {
      const int* rr = p.inj_row + (size_t)t * (TY + 1);
      const int r1 = rr[ly + 1];
      for (int e = rr[ly]; e < r1; ++e) {
        const int elx = p.inj_loc[e] - ly * TX;
        if ((elx >> 2) == tx) {
          const float val = p.inj_scale * p.inj_w[e] * p.vals[p.inj_vidx[e] + p.step_off];
          const int ix = elx & 3;
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] += (q == ix) ? val : 0.f;
        }
      }
    }
  }

  // epilogue on the float4 of points (lanes outside the grid keep the padding at 0)
  bool in[4];
#pragma unroll
  for (int ix = 0; ix < 4; ++ix) in[ix] = (yg < p.ny) && (xg + ix < p.nx);
  float k[4], a0[4];
  unpack(ldg4(p.kf + pi), k);
  {
    float ax[4];
    unpack(ldg4(p.spx + xg), ax);
    const float ay = p.spy[yg];
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) a0[ix] = ax[ix] + ay;
  }
  float* upp = p.up + fo + pi;
  if (MODE == EXT_KW) {
    float o[4];
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) o[ix] = in[ix] ? k[ix] * acc[ix] : 0.f;
    st4(p.out + fo + pi, pack(o));
    return;
  }
  float uo[4], r[4];
  unpack(ld4(upp), uo);
  if (MODE == EXT_T4) {
    float uc[4], F[4];
    unpack(ld4(p.u + fo + pi), uc);
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) {
      F[ix] = fmaf(k[ix] * acc[ix], INV12, cen[ix]);
      r[ix] = in[ix] ? (2.f * uc[ix] - (1.f - a0[ix]) * uo[ix] + F[ix]) * __frcp_rn(1.f + a0[ix]) : 0.f;
    }
    st4(upp, pack(r));
    if (!ADJ) {
      if (p.hist) {
        float f[4], w[4];
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) {
          f[ix] = in[ix] ? F[ix] : 0.f;
          w[ix] = in[ix] ? cen[ix] : 0.f;
        }
        __stcs(reinterpret_cast<float4*>(p.hist + fo + pi), pack(f));
        __stcs(reinterpret_cast<float4*>(p.hist2 + fo + pi), pack(w));
      }
    } else if (p.image) {
      float h[4], h2[4], g[4];
      unpack(__ldcs(reinterpret_cast<const float4*>(p.hist + fo + pi)), h);
      unpack(__ldcs(reinterpret_cast<const float4*>(p.hist2 + fo + pi)), h2);
      unpack(ld4(p.g + fo + pi), g);
#pragma unroll
      for (int ix = 0; ix < 4; ++ix)
        if (in[ix]) g[ix] = g[ix] - fmaf(cen[ix] * h2[ix], INV12, uc[ix] * h[ix]);
      st4(p.g + fo + pi, pack(g));
    }
    return;
  }
  float at[4], hh[4];
  unpack(ldg4(p.att + pi), at);
  if (MODE == EXT_ATT0) {
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) {
      const float a = a0[ix] + at[ix];
      const float h = k[ix] * acc[ix];
      const float rv = (2.f * cen[ix] - (1.f - a) * uo[ix] + h) * __frcp_rn(1.f + a);
      r[ix] = in[ix] ? rv : 0.f;
      hh[ix] = in[ix] ? h - 0.5f * at[ix] * (rv - uo[ix]) : 0.f;
    }
  } else {   // EXT_ATT2
    float qv[4], qn[4];
    unpack(ld4(p.q + fo + pi), qv);
#pragma unroll
    for (int ix = 0; ix < 4; ++ix) {
      float E, extra = 0.f;
      if (!ADJ) {
        const float dl = lap[ix] - qv[ix];
        E = fmaf(at[ix], dl, acc[ix]);
        qn[ix] = lap[ix];
        extra = 0.5f * k[ix] * at[ix] * dl;
      } else {
        E = acc[ix] + (lc[ix] - qv[ix]);
        qn[ix] = lc[ix];
      }
      const float h = k[ix] * E;
      const float rv = (2.f * cen[ix] - (1.f - a0[ix]) * uo[ix] + h) * __frcp_rn(1.f + a0[ix]);
      r[ix] = in[ix] ? rv : 0.f;
      hh[ix] = in[ix] ? h + extra : 0.f;
      qn[ix] = in[ix] ? qn[ix] : 0.f;
    }
    st4(p.q + fo + pi, pack(qn));
  }
  st4(upp, pack(r));
  if (!ADJ) {
    if (p.hist) __stcs(reinterpret_cast<float4*>(p.hist + fo + pi), pack(hh));
  } else if (p.image) {
    float h[4], g[4];
    unpack(__ldcs(reinterpret_cast<const float4*>(p.hist + fo + pi)), h);
    unpack(ld4(p.g + fo + pi), g);
#pragma unroll
    for (int ix = 0; ix < 4; ++ix)
      if (in[ix]) g[ix] = fmaf(-cen[ix], h[ix], g[ix]);
    st4(p.g + fo + pi, pack(g));
  }
}

template <int R, bool VD, bool ADJ, int MODE>
__global__ void __launch_bounds__(EXT_TX * EXT_TY3, 3) k_ext3d(const StepParams p) {
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
    sample_receivers(p, blk * NT + tid);
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
  // each plane scans only its own injection entries
  __shared__ int s_pe[MAX_ZCHUNK + 1];
  const bool has_inj = p.inj_off && p.inj_off[tile + 1] > p.inj_off[tile];
  if (has_inj) plane_entries(p, tile, z1 - z0, TY * TX, tid, NT, s_pe);

  for (int z = z0; z < z1; ++z) {
    const long long pz = (long long)(z + p.oz) * p.sxy;
    const long long idx = col + pz;
    PointOps<VD, ADJ, MODE> ops;
    if (in_xy) ops.load(p, fo, idx);
    {
      const long long o = col + pz + (long long)R * p.sxy;
      q[Q - 1] = X[o];
      if (PSI) qz[Q - 1] = __ldg(p.bz + o) * q[Q - 1];
      if (CL) qc[Q - 1] = __ldg(p.att + o) * q[Q - 1];
    }
    __syncthreads();   // the previous plane's readers are done with the shared tiles
    const long long pb = pz + (long long)(y0 + p.oy - R) * p.sx + (x0 + p.ox - R);
    // fixed trip counts, unrolled: every thread's loads of the plane issue together
#pragma unroll
    for (int t = 0; t < (SH * SW + NT - 1) / NT; ++t) {
      const int i = tid + t * NT;
      if (i < SH * SW) {
        const int r = i / SW, c = i - r * SW;
        const long long o = pb + (long long)r * p.sx + c;
        const float v = X[o];
        s_x[r][c] = v;
        if (CL) s_c[r][c] = __ldg(p.att + o) * v;
      }
    }
    if (PSI) {
#pragma unroll
      for (int t = 0; t < (TY * SW + NT - 1) / NT; ++t) {
        const int i = tid + t * NT;
        if (i < TY * SW) {
          const int r = i / SW, c = i - r * SW;
          const long long o = pb + (long long)(r + R) * p.sx + c;
          s_px[r][c] = __ldg(p.bx + o) * X[o];
        }
      }
#pragma unroll
      for (int t = 0; t < (SH * TX + NT - 1) / NT; ++t) {
        const int i = tid + t * NT;
        if (i < SH * TX) {
          const int r = i / TX, c = i - r * TX;
          const long long o = pb + (long long)r * p.sx + c + R;
          s_py[r][c] = __ldg(p.by + o) * X[o];
        }
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
    if (VD && !ADJ) {
      float dx = 0.f, dy = 0.f, dz = 0.f;
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        dx = fmaf(p.wx.w1[j], s_x[cy][cx + j] - s_x[cy][cx - j], dx);
        dy = fmaf(p.wy.w1[j], s_x[cy + j][cx] - s_x[cy - j][cx], dy);
        dz = fmaf(p.wz.w1[j], q[R + j] - q[R - j], dz);
      }
      acc -= ops.bx * dx + ops.by * dy + ops.bz * dz;
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
    if (has_inj) {
      const int lz = z - z0, loc = (lz * TY + ty) * TX + tx;
      for (int e = s_pe[lz], e1 = s_pe[lz + 1]; e < e1; ++e)
        if (p.inj_loc[e] == loc)
          acc = fmaf(p.inj_scale * p.inj_w[e], p.vals[p.inj_vidx[e] + p.step_off], acc);
    }
    if (in_xy) ext_update<VD, ADJ, MODE>(p, fo, idx, cen, acc, lap, lc, axy + p.spz[z], ops);
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
    constexpr size_t smem = Ext2<R, VD, ADJ, MODE>::SMEM;
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(k_ext2d<R, VD, ADJ, MODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
    dim3 grid((p.nx + EXT_TX2 - 1) / EXT_TX2, (p.ny + EXT_TY2 - 1) / EXT_TY2, p.B);
    k_ext2d<R, VD, ADJ, MODE><<<grid, dim3(EXT_TX2 / 4, EXT_TY2), smem, st>>>(p);
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
                           float* __restrict__ g, long long fs, int nb, int S) {
  // slot b images into gradient slot b / S (S shots per CTA in the step kernels)
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < fs;
       i += (long long)gridDim.x * blockDim.x) {
    for (int b = 0; b < nb; ++b) {
      const long long o = (long long)b * fs + i;
      const long long og = (long long)(b / S) * fs + i;
      g[og] = g[og] - fmaf(ky[o] * kw[o], INV12, lam[o] * F[o]);
    }
  }
}

}  // namespace

cudaError_t launch_image_t4(const Layout& L, const float* lam, const float* ky, const float* F,
                            const float* kw, float* g, int nb, int S, cudaStream_t st) {
  const long long fs = L.fstride;
  long long blocks = (fs + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  k_image_t4<<<(int)blocks, 256, 0, st>>>(lam, ky, F, kw, g, fs, nb, S);
  return cudaGetLastError();
}

}  // namespace fwi
