// Perfectly matched layer (Sec. 2.4 offers a PML next to the sponge): the
// unsplit second-order form from the coordinate stretching
// d_j -> d_j / (1 + z_j / p), with the sponge's per-axis profiles z_j.  With
// A_j = z_j dt / 2 (the sponge arrays), k = (vp dt)^2,
//   a = sum A,  e = 4 (A_x A_y + A_x A_z + A_y A_z),  f = 8 A_x A_y A_z / dt,
//   p_j = (1 - A_j) / (1 + A_j),  b_j = 2 (A_k + A_l - A_j) / (1 + A_j),
//   g_j = 4 A_k A_l / (dt (1 + A_j))      (k, l the other axes; A_z = 0 in 2D)
// one time step is
//   PML_U:   E = L u^n + s^n + sum_j D1_j phi_j^n,
//            (1+a) u^{n+1} = 2u^n - (1-a) u^{n-1} - e u^n - f q^n + k E,
//            q^{n+1} = q^n + dt u^{n+1}   (3D),   h^n = k E stored;
//   PML_PHI: phi_j^{n+1} = p_j phi_j^n + b_j D1_j u^{n+1} + g_j D1_j q^{n+1},
// (D1 the solver's first-derivative stencil; outside the layer every A is 0,
// phi stays 0 and PML_U is the leapfrog, so PML_PHI skips tiles that do not
// touch the layer).  The exact discrete adjoint runs backwards, per step n:
//   PML_A:   ub = ubar^{n+1} - sum_j D1_j(b_j phibar_j) + dt qb,
//            qb = qbar^{n+1} - sum_j D1_j(g_j phibar_j),  c^n = ub / (1+a),
//            qbar^n = qb - f c^n,  ubar^{n-1} = P^T r^{n-1} - (1-a) c^n,
//            g -= (k c^n) h^n   (the imaging condition of Sec. 2.2, Eq. 8);
//   PML_B:   ubar^n += (2 - e) c^n + L^T(k c^n),
//            phibar_j^n = p_j phibar_j^{n+1} - D1_j(k c^n).
// 2D: a CTA of 32 x 16 threads on a 128 x 16 tile, a float4 of x points per
// thread.  3D: a CTA of 32 x 8 threads streaming a column along z with the
// column's values in register queues, one point per thread.
#include "fwi_internal.cuh"

namespace fwi {

namespace {

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

// A_j at index i of an axis of n points (0 outside the grid).
__device__ __forceinline__ float sp_at(const float* sp, int i, int n) {
  return (i >= 0 && i < n) ? sp[i] : 0.f;
}
// b_j and g_j of axis j from A_j and the other two axes' A_k, A_l.
__device__ __forceinline__ float pml_b(float Aj, float Ak, float Al) {
  return 2.f * ((Ak + Al) - Aj) / (1.f + Aj);
}
__device__ __forceinline__ float pml_g(float Aj, float Ak, float Al, float dt) {
  return 4.f * Ak * Al / (dt * (1.f + Aj));
}
__device__ __forceinline__ float pml_p(float Aj) { return (1.f - Aj) / (1.f + Aj); }


template <int R>
struct Pml2 {
  static constexpr int TX = EXT_TX2, TY = EXT_TY2;
  static constexpr int XH = (R <= 4) ? 4 : 8, NL = XH / 4;
  static constexpr int SW = TX / 4 + 2 * NL, SH = TY + 2 * R, QW = TX / 4;
  static constexpr size_t SMEM = ((size_t)SH * SW + TY * SW + SH * QW) * 16;
};

template <int R, bool VD, int MODE>
__global__ void __launch_bounds__(EXT_TX2 / 4 * EXT_TY2, 2) k_pml2d(const StepParams p) {
  using G = Pml2<R>;
  constexpr int TX = G::TX, TY = G::TY, NL = G::NL, SW = G::SW, SH = G::SH, QW = G::QW;
  constexpr int XH = G::XH;
  constexpr int NT = TX / 4 * TY;
  constexpr int NV = 4 + 8 * NL;
  constexpr bool FULL = MODE != PML_A;     // the stencil input tile with halo
  constexpr bool CROSS = MODE == PML_U || MODE == PML_A || (MODE == PML_B && VD);
  extern __shared__ __align__(16) float4 sm[];
  float4* s_x = sm;                        // [SH][SW]
  float4* s_r = sm + SH * SW;              // tile rows with x halo [TY][SW]
  float4* s_c = s_r + TY * SW;             // tile columns with y halo [SH][QW]

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * (TX / 4) + tx;
  const int b = blockIdx.z;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const long long fo = (long long)b * p.fstride;
  if (MODE == PML_PHI) {   // phi changes only inside the layer
    if (!(x0 < p.nb || x0 + TX > p.nx - p.nb || y0 < p.nb || y0 + TY > p.ny - p.nb)) return;
  }
  // phi (phibar) matter only in the layer and are read within R of it: tiles
  // farther away skip them (phi is 0 there; phibar is never read there)
  const int reach = p.nb + R;
  const bool near = x0 < reach || x0 + TX > p.nx - reach || y0 < reach || y0 + TY > p.ny - reach;
  if (MODE == PML_U) {
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    sample_receivers(p, blk * NT + tid);
  }
  const float* __restrict__ X = p.x + fo;
  const long long base = (long long)(y0 + p.oy - R) * p.sx + (x0 + p.ox - XH);
  if (FULL) {
    for (int i = tid; i < SH * SW; i += NT) {
      const int r = i / SW, c = i - r * SW;
      const long long o = base + (long long)r * p.sx + 4 * c;
      const float4 xv = ldg4(X + o);
      s_x[i] = (MODE == PML_B) ? mul4(ldg4(p.kf + o), xv) : xv;
    }
  }
  const bool cross = CROSS && (near || MODE == PML_B);
  if (cross) {
    for (int i = tid; i < TY * SW; i += NT) {
      const int r = i / SW, c = i - r * SW;
      const long long o = base + (long long)(r + R) * p.sx + 4 * c;
      if (MODE == PML_U) {
        s_r[i] = ldg4(p.ph[0] + fo + o);
      } else if (MODE == PML_A) {     // b_x phibar_x
        float f[4];
        unpack(ldg4(p.ph[0] + fo + o), f);
        const float Ay = sp_at(p.spy, y0 + r, p.ny);
#pragma unroll
        for (int l = 0; l < 4; ++l) f[l] *= pml_b(sp_at(p.spx, x0 - XH + 4 * c + l, p.nx), Ay, 0.f);
        s_r[i] = pack(f);
      } else {                        // b_x k c
        s_r[i] = mul4(ldg4(p.bx + o), mul4(ldg4(p.kf + o), ldg4(X + o)));
      }
    }
    for (int i = tid; i < SH * QW; i += NT) {
      const int r = i / QW, c = i - r * QW;
      const long long o = base + (long long)r * p.sx + 4 * (c + NL);
      if (MODE == PML_U) {
        s_c[i] = ldg4(p.ph[1] + fo + o);
      } else if (MODE == PML_A) {     // b_y phibar_y
        float f[4];
        unpack(ldg4(p.ph[1] + fo + o), f);
        const float Ay = sp_at(p.spy, y0 - R + r, p.ny);
#pragma unroll
        for (int l = 0; l < 4; ++l) f[l] *= pml_b(Ay, sp_at(p.spx, x0 + 4 * c + l, p.nx), 0.f);
        s_c[i] = pack(f);
      } else {                        // b_y k c
        s_c[i] = mul4(ldg4(p.by + o), mul4(ldg4(p.kf + o), ldg4(X + o)));
      }
    }
  }
  __syncthreads();

  const int ly = ty, yg = y0 + ly, srow = ly + R;
  const int xg = x0 + 4 * tx;
  const long long pi = (long long)(yg + p.oy) * p.sx + (xg + p.ox);
  bool in[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) in[l] = (yg < p.ny) && (xg + l < p.nx);
  float Ax[4];
  unpack(ldg4(p.spx + xg), Ax);
  const float Ay = p.spy[yg];

  float v[NV], cen[4] = {0.f, 0.f, 0.f, 0.f}, acc[4] = {0.f, 0.f, 0.f, 0.f};
  float d1x[4] = {0.f, 0.f, 0.f, 0.f}, d1y[4] = {0.f, 0.f, 0.f, 0.f};
  if (FULL) {
#pragma unroll
    for (int q = 0; q <= 2 * NL; ++q) unpack(s_x[srow * SW + tx + q], v + 4 * q);
    float c2[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int c = 4 * NL + l;
      cen[l] = v[c];
      c2[l] = v[c] + v[c];
      if (MODE != PML_PHI) {
#pragma unroll
        for (int j = 1; j <= R; ++j) acc[l] = fmaf(p.wx.w2[j], (v[c + j] + v[c - j]) - c2[l], acc[l]);
      }
#pragma unroll
      for (int j = 1; j <= R; ++j) d1x[l] = fmaf(p.wx.w1[j], v[c + j] - v[c - j], d1x[l]);
    }
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      float a[4], cc[4];
      unpack(s_x[(srow - j) * SW + tx + NL], a);
      unpack(s_x[(srow + j) * SW + tx + NL], cc);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        if (MODE != PML_PHI) acc[l] = fmaf(p.wy.w2[j], (a[l] + cc[l]) - c2[l], acc[l]);
        d1y[l] = fmaf(p.wy.w1[j], cc[l] - a[l], d1y[l]);
      }
    }
  }
  if (MODE == PML_U && VD) {   // L_rho u = lap u - b . grad u
    float bxv[4], byv[4];
    unpack(ldg4(p.bx + pi), bxv);
    unpack(ldg4(p.by + pi), byv);
#pragma unroll
    for (int l = 0; l < 4; ++l) acc[l] -= bxv[l] * d1x[l] + byv[l] * d1y[l];
  }
  // D1x of the row tile and D1y of the column tile: phi (PML_U), b phibar
  // (PML_A), b k c (PML_B, variable density)
  float dr[4] = {0.f, 0.f, 0.f, 0.f};
  if (cross) {
    float w[NV];
#pragma unroll
    for (int q = 0; q <= 2 * NL; ++q) unpack(s_r[ly * SW + tx + q], w + 4 * q);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int c = 4 * NL + l;
#pragma unroll
      for (int j = 1; j <= R; ++j) dr[l] = fmaf(p.wx.w1[j], w[c + j] - w[c - j], dr[l]);
    }
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      float a[4], cc[4];
      unpack(s_c[(srow - j) * QW + tx], a);
      unpack(s_c[(srow + j) * QW + tx], cc);
#pragma unroll
      for (int l = 0; l < 4; ++l) dr[l] = fmaf(p.wy.w1[j], cc[l] - a[l], dr[l]);
    }
  }
  // sources (PML_U) or the residual of step n-1 (PML_A): this row's entries
  float inj[4] = {0.f, 0.f, 0.f, 0.f};
  if ((MODE == PML_U || MODE == PML_A) && p.inj_off) {
    const int t = b * p.ntiles + blockIdx.y * gridDim.x + blockIdx.x;
    if (p.inj_off[t + 1] > p.inj_off[t]) {
      const int* rr = p.inj_row + (size_t)t * (TY + 1);
      const int r1 = rr[ly + 1];
      for (int e = rr[ly]; e < r1; ++e) {
        const int elx = p.inj_loc[e] - ly * TX;
        if ((elx >> 2) == tx) {
          const float val = p.inj_w[e] * p.vals[p.inj_vidx[e] + p.step_off];
          const int l = elx & 3;
#pragma unroll
          for (int q = 0; q < 4; ++q) inj[q] += (q == l) ? val : 0.f;
        }
      }
    }
  }

  if (MODE == PML_U) {
    float k[4], uo[4], r[4], h[4];
    unpack(ldg4(p.kf + pi), k);
    unpack(ld4(p.up + fo + pi), uo);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const float E = (acc[l] + inj[l]) + dr[l];
      const float a = Ax[l] + Ay;
      const float e = 4.f * Ax[l] * Ay;
      const float hv = k[l] * E;
      const float rv = (2.f * cen[l] - (1.f - a) * uo[l] - e * cen[l] + hv) / (1.f + a);
      r[l] = in[l] ? rv : 0.f;
      h[l] = in[l] ? hv : 0.f;
    }
    st4(p.up + fo + pi, pack(r));
    if (p.hist) __stcs(reinterpret_cast<float4*>(p.hist + fo + pi), pack(h));
  } else if (MODE == PML_PHI) {
    float fx[4], fy[4];
    unpack(ld4(p.ph[0] + fo + pi), fx);
    unpack(ld4(p.ph[1] + fo + pi), fy);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const float nx_ = pml_p(Ax[l]) * fx[l] + pml_b(Ax[l], Ay, 0.f) * d1x[l];
      const float ny_ = pml_p(Ay) * fy[l] + pml_b(Ay, Ax[l], 0.f) * d1y[l];
      fx[l] = in[l] ? nx_ : 0.f;
      fy[l] = in[l] ? ny_ : 0.f;
    }
    st4(p.ph[0] + fo + pi, pack(fx));
    st4(p.ph[1] + fo + pi, pack(fy));
  } else if (MODE == PML_A) {
    float k[4], xn[4], h[4], g[4], cc[4], un[4];
    unpack(ldg4(p.kf + pi), k);
    unpack(ld4(p.up + fo + pi), xn);
    unpack(__ldcs(reinterpret_cast<const float4*>(p.hist + fo + pi)), h);
    unpack(ld4(p.g + fo + pi), g);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const float a = Ax[l] + Ay;
      const float c = (xn[l] - dr[l]) / (1.f + a);
      cc[l] = in[l] ? c : 0.f;
      un[l] = in[l] ? inj[l] - (1.f - a) * c : 0.f;
      if (in[l]) g[l] = fmaf(-(k[l] * c), h[l], g[l]);
    }
    st4(p.out + fo + pi, pack(cc));
    st4(p.up + fo + pi, pack(un));
    st4(p.g + fo + pi, pack(g));
  } else {   // PML_B
    float c[4], xc[4];
    unpack(ld4(p.x + fo + pi), c);
    unpack(ld4(p.up + fo + pi), xc);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const float e = 4.f * Ax[l] * Ay;
      const float LT = acc[l] + (VD ? dr[l] : 0.f);
      const float nxc = xc[l] + ((2.f - e) * c[l] + LT);
      xc[l] = in[l] ? nxc : 0.f;
    }
    st4(p.up + fo + pi, pack(xc));
    if (near) {
      float fx[4], fy[4];
      unpack(ld4(p.ph[0] + fo + pi), fx);
      unpack(ld4(p.ph[1] + fo + pi), fy);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const float nfx = pml_p(Ax[l]) * fx[l] - d1x[l];
        const float nfy = pml_p(Ay) * fy[l] - d1y[l];
        fx[l] = in[l] ? nfx : 0.f;
        fy[l] = in[l] ? nfy : 0.f;
      }
      st4(p.ph[0] + fo + pi, pack(fx));
      st4(p.ph[1] + fo + pi, pack(fy));
    }
  }
}

// 3D: 32 x 8 columns streamed along z, one point per thread.
template <int R, bool VD, int MODE>
__global__ void __launch_bounds__(EXT_TX * EXT_TY3, 3) k_pml3d(const StepParams p) {
  constexpr int TX = EXT_TX, TY = EXT_TY3;
  constexpr int SW = TX + 2 * R, SH = TY + 2 * R;
  constexpr int NT = TX * TY;
  constexpr int Q = 2 * R + 1;
  constexpr bool FULL = MODE != PML_A;                     // stencil input plane (all axes)
  constexpr bool QQ = MODE == PML_PHI;                     // q^{n+1} plane (all axes)
  constexpr bool CROSS = MODE == PML_U || MODE == PML_A || (MODE == PML_B && VD);
  constexpr bool CROSS2 = MODE == PML_A;                   // g phibar
  __shared__ float s_x[FULL ? SH : 1][FULL ? SW : 1];
  __shared__ float s_q[QQ ? SH : 1][QQ ? SW : 1];
  __shared__ float s_r[CROSS ? TY : 1][CROSS ? SW : 1];
  __shared__ float s_c[CROSS ? SH : 1][CROSS ? TX : 1];
  __shared__ float s_r2[CROSS2 ? TY : 1][CROSS2 ? SW : 1];
  __shared__ float s_c2[CROSS2 ? SH : 1][CROSS2 ? TX : 1];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int b = blockIdx.z / p.nzc;
  const int zc = blockIdx.z - b * p.nzc;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = zc * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.nz);
  const long long fo = (long long)b * p.fstride;
  if (MODE == PML_PHI) {
    if (!(x0 < p.nb || x0 + TX > p.nx - p.nb || y0 < p.nb || y0 + TY > p.ny - p.nb ||
          z0 < p.nb || z1 > p.nz - p.nb))
      return;
  }
  const int reach = p.nb + R;
  const bool near = x0 < reach || x0 + TX > p.nx - reach || y0 < reach || y0 + TY > p.ny - reach ||
                    z0 < reach || z1 > p.nz - reach;
  const bool cross = CROSS && (near || MODE == PML_B);
  if (MODE == PML_U) {
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    sample_receivers(p, blk * NT + tid);
  }
  const float* __restrict__ X = p.x + fo;
  const int xg = x0 + tx, yg = y0 + ty;
  const long long col = (long long)(yg + p.oy) * p.sx + (xg + p.ox);
  const float Ax = sp_at(p.spx, xg, p.nx), Ay = sp_at(p.spy, yg, p.ny);
  const bool in_xy = (xg < p.nx) && (yg < p.ny);
  const int tile = b * p.ntiles + (zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int cx = tx + R, cy = ty + R;
  // each plane scans only its own injection entries
  __shared__ int s_pe[MAX_ZCHUNK + 1];
  const bool has_inj = (MODE == PML_U || MODE == PML_A) && p.inj_off &&
                       p.inj_off[tile + 1] > p.inj_off[tile];
  if (has_inj) plane_entries(p, tile, z1 - z0, TY * TX, tid, NT, s_pe);

  // z queues of this column: the stencil input (kc in PML_B); phi_z (PML_U);
  // q (PML_PHI); b_z phibar_z and g_z phibar_z (PML_A); b_z k c (PML_B, vd)
  float q1[Q], q2[Q], q3[Q];
  auto col_vals = [&](int zz, float& v1, float& v2, float& v3) {
    const long long o = col + (long long)(zz + p.oz) * p.sxy;
    const float Az = sp_at(p.spz, zz, p.nz);
    v1 = v2 = v3 = 0.f;
    if (FULL) v1 = (MODE == PML_B) ? __ldg(p.kf + o) * X[o] : X[o];
    if (MODE == PML_U && near) v2 = p.ph[2][fo + o];
    if (MODE == PML_PHI) v2 = p.q[fo + o];
    if (MODE == PML_A && near) {
      const float f = p.ph[2][fo + o];
      v2 = pml_b(Az, Ax, Ay) * f;
      v3 = pml_g(Az, Ax, Ay, p.dt) * f;
    }
    if (MODE == PML_B && VD) v2 = __ldg(p.bz + o) * v1;
  };
#pragma unroll
  for (int j = 0; j < Q - 1; ++j) col_vals(z0 - R + j, q1[j], q2[j], q3[j]);

  for (int z = z0; z < z1; ++z) {
    const long long pz = (long long)(z + p.oz) * p.sxy;
    const long long idx = col + pz;
    // the point's own operands (read and written by this thread only), loaded
    // ahead of the plane staging, the barrier and the stencil
    float o_k = 0.f, o_up = 0.f, o_q = 0.f, o_h = 0.f, o_g = 0.f, o_c = 0.f;
    float o_b[3] = {0.f, 0.f, 0.f}, o_f[3] = {0.f, 0.f, 0.f};
    if (in_xy) {
      if (MODE != PML_PHI) o_k = __ldg(p.kf + idx);
      if (MODE != PML_PHI) o_up = p.up[fo + idx];
      if (MODE == PML_U || MODE == PML_A) o_q = p.q[fo + idx];
      if (MODE == PML_U && VD) {
        o_b[0] = __ldg(p.bx + idx);
        o_b[1] = __ldg(p.by + idx);
        o_b[2] = __ldg(p.bz + idx);
      }
      if (MODE == PML_A) {
        o_h = __ldcs(p.hist + fo + idx);
        o_g = p.g[fo + idx];
      }
      if (MODE == PML_B) o_c = X[idx];
      if (MODE == PML_PHI || (MODE == PML_B && near)) {
#pragma unroll
        for (int j = 0; j < 3; ++j) o_f[j] = p.ph[j][fo + idx];
      }
    }
    col_vals(z + R, q1[Q - 1], q2[Q - 1], q3[Q - 1]);
    const float Az = sp_at(p.spz, z, p.nz);
    __syncthreads();   // the previous plane's readers are done with the shared tiles
    const long long pb = pz + (long long)(y0 + p.oy - R) * p.sx + (x0 + p.ox - R);
    // fixed trip counts, unrolled: every thread's loads of the plane issue together
    if (FULL || QQ) {
#pragma unroll
      for (int t = 0; t < (SH * SW + NT - 1) / NT; ++t) {
        const int i = tid + t * NT;
        if (i >= SH * SW) break;
        const int r = i / SW, c = i - r * SW;
        const long long o = pb + (long long)r * p.sx + c;
        if (FULL) s_x[r][c] = (MODE == PML_B) ? __ldg(p.kf + o) * X[o] : X[o];
        if (QQ) s_q[r][c] = p.q[fo + o];
      }
    }
    if (cross) {
#pragma unroll
      for (int t = 0; t < (TY * SW + NT - 1) / NT; ++t) {
        const int i = tid + t * NT;
        if (i >= TY * SW) break;
        const int r = i / SW, c = i - r * SW;
        const long long o = pb + (long long)(r + R) * p.sx + c;
        if (MODE == PML_U) {
          s_r[r][c] = p.ph[0][fo + o];
        } else if (MODE == PML_A) {
          const float f = p.ph[0][fo + o];
          const float ax = sp_at(p.spx, x0 - R + c, p.nx), ay = sp_at(p.spy, y0 + r, p.ny);
          s_r[r][c] = pml_b(ax, ay, Az) * f;
          s_r2[r][c] = pml_g(ax, ay, Az, p.dt) * f;
        } else {
          s_r[r][c] = __ldg(p.bx + o) * __ldg(p.kf + o) * X[o];
        }
      }
#pragma unroll
      for (int t = 0; t < (SH * TX + NT - 1) / NT; ++t) {
        const int i = tid + t * NT;
        if (i >= SH * TX) break;
        const int r = i / TX, c = i - r * TX;
        const long long o = pb + (long long)r * p.sx + c + R;
        if (MODE == PML_U) {
          s_c[r][c] = p.ph[1][fo + o];
        } else if (MODE == PML_A) {
          const float f = p.ph[1][fo + o];
          const float ay = sp_at(p.spy, y0 - R + r, p.ny), ax = sp_at(p.spx, x0 + c, p.nx);
          s_c[r][c] = pml_b(ay, ax, Az) * f;
          s_c2[r][c] = pml_g(ay, ax, Az, p.dt) * f;
        } else {
          s_c[r][c] = __ldg(p.by + o) * __ldg(p.kf + o) * X[o];
        }
      }
    }
    __syncthreads();

    float cen = 0.f, acc = 0.f, d1x = 0.f, d1y = 0.f, d1z = 0.f;
    if (FULL) {
      cen = q1[R];
      const float c2 = cen + cen;
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        if (MODE != PML_PHI) {
          acc = fmaf(p.wx.w2[j], (s_x[cy][cx + j] + s_x[cy][cx - j]) - c2, acc);
          acc = fmaf(p.wy.w2[j], (s_x[cy + j][cx] + s_x[cy - j][cx]) - c2, acc);
          acc = fmaf(p.wz.w2[j], (q1[R + j] + q1[R - j]) - c2, acc);
        }
        d1x = fmaf(p.wx.w1[j], s_x[cy][cx + j] - s_x[cy][cx - j], d1x);
        d1y = fmaf(p.wy.w1[j], s_x[cy + j][cx] - s_x[cy - j][cx], d1y);
        d1z = fmaf(p.wz.w1[j], q1[R + j] - q1[R - j], d1z);
      }
    }
    if (MODE == PML_U && VD)
      acc -= o_b[0] * d1x + o_b[1] * d1y + o_b[2] * d1z;
    float dr = 0.f, dr2 = 0.f;   // D1 of the cross tiles and queues
    if (cross) {
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        dr = fmaf(p.wx.w1[j], s_r[ty][cx + j] - s_r[ty][cx - j], dr);
        dr = fmaf(p.wy.w1[j], s_c[cy + j][tx] - s_c[cy - j][tx], dr);
        if (MODE != PML_B || VD) dr = fmaf(p.wz.w1[j], q2[R + j] - q2[R - j], dr);
        if (CROSS2) {
          dr2 = fmaf(p.wx.w1[j], s_r2[ty][cx + j] - s_r2[ty][cx - j], dr2);
          dr2 = fmaf(p.wy.w1[j], s_c2[cy + j][tx] - s_c2[cy - j][tx], dr2);
          dr2 = fmaf(p.wz.w1[j], q3[R + j] - q3[R - j], dr2);
        }
      }
    }
    float inj = 0.f;
    if (has_inj) {
      const int lz = z - z0, loc = (lz * TY + ty) * TX + tx;
      for (int e = s_pe[lz], e1 = s_pe[lz + 1]; e < e1; ++e)
        if (p.inj_loc[e] == loc) inj += p.inj_w[e] * p.vals[p.inj_vidx[e] + p.step_off];
    }
    if (in_xy) {
      const float k = o_k;
      const float a = Ax + Ay + Az;
      const float e = 4.f * (Ax * Ay + Ax * Az + Ay * Az);
      const float f = 8.f * Ax * Ay * Az / p.dt;
      if (MODE == PML_U) {
        const float E = (acc + inj) + dr;
        const float hv = k * E;
        const float uo = o_up;
        const float qv = o_q;
        const float r = (2.f * cen - (1.f - a) * uo - e * cen - f * qv + hv) / (1.f + a);
        p.up[fo + idx] = r;
        p.q[fo + idx] = qv + p.dt * r;
        if (p.hist) __stcs(p.hist + fo + idx, hv);
      } else if (MODE == PML_PHI) {
        float dqx = 0.f, dqy = 0.f, dqz = 0.f;
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          dqx = fmaf(p.wx.w1[j], s_q[cy][cx + j] - s_q[cy][cx - j], dqx);
          dqy = fmaf(p.wy.w1[j], s_q[cy + j][cx] - s_q[cy - j][cx], dqy);
          dqz = fmaf(p.wz.w1[j], q2[R + j] - q2[R - j], dqz);
        }
        float* fx = p.ph[0] + fo + idx;
        float* fy = p.ph[1] + fo + idx;
        float* fz = p.ph[2] + fo + idx;
        *fx = pml_p(Ax) * o_f[0] + pml_b(Ax, Ay, Az) * d1x + pml_g(Ax, Ay, Az, p.dt) * dqx;
        *fy = pml_p(Ay) * o_f[1] + pml_b(Ay, Ax, Az) * d1y + pml_g(Ay, Ax, Az, p.dt) * dqy;
        *fz = pml_p(Az) * o_f[2] + pml_b(Az, Ax, Ay) * d1z + pml_g(Az, Ax, Ay, p.dt) * dqz;
      } else if (MODE == PML_A) {
        const float qb = o_q - dr2;
        const float ub = (o_up - dr) + p.dt * qb;
        const float c = ub / (1.f + a);
        p.q[fo + idx] = qb - f * c;
        p.out[fo + idx] = c;
        p.up[fo + idx] = inj - (1.f - a) * c;
        p.g[fo + idx] = fmaf(-(k * c), o_h, o_g);
      } else {   // PML_B
        const float c = o_c;
        const float LT = acc + (VD ? dr : 0.f);
        p.up[fo + idx] = o_up + ((2.f - e) * c + LT);
        if (near) {
          p.ph[0][fo + idx] = pml_p(Ax) * o_f[0] - d1x;
          p.ph[1][fo + idx] = pml_p(Ay) * o_f[1] - d1y;
          p.ph[2][fo + idx] = pml_p(Az) * o_f[2] - d1z;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < Q - 1; ++j) {
      q1[j] = q1[j + 1];
      q2[j] = q2[j + 1];
      q3[j] = q3[j + 1];
    }
  }
}

template <int R, bool VD, int MODE>
cudaError_t launch_m(const StepParams& p, int ndim, cudaStream_t st) {
  if (ndim == 2) {
    constexpr size_t smem = Pml2<R>::SMEM;
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(k_pml2d<R, VD, MODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
    dim3 grid((p.nx + EXT_TX2 - 1) / EXT_TX2, (p.ny + EXT_TY2 - 1) / EXT_TY2, p.B);
    k_pml2d<R, VD, MODE><<<grid, dim3(EXT_TX2 / 4, EXT_TY2), smem, st>>>(p);
  } else {
    dim3 grid((p.nx + EXT_TX - 1) / EXT_TX, (p.ny + EXT_TY3 - 1) / EXT_TY3, p.B * p.nzc);
    k_pml3d<R, VD, MODE><<<grid, dim3(EXT_TX, EXT_TY3), 0, st>>>(p);
  }
  return cudaGetLastError();
}

template <int R, bool VD>
cudaError_t launch_mode(const StepParams& p, int ndim, int mode, cudaStream_t st) {
  switch (mode) {
    case PML_U: return launch_m<R, VD, PML_U>(p, ndim, st);
    case PML_PHI: return launch_m<R, VD, PML_PHI>(p, ndim, st);
    case PML_A: return launch_m<R, VD, PML_A>(p, ndim, st);
    default: return launch_m<R, VD, PML_B>(p, ndim, st);
  }
}

}  // namespace

cudaError_t launch_pml(const StepParams& p, int ndim, int R, bool vd, int mode, cudaStream_t st) {
  if (R == 4) return vd ? launch_mode<4, true>(p, ndim, mode, st) : launch_mode<4, false>(p, ndim, mode, st);
  return vd ? launch_mode<5, true>(p, ndim, mode, st) : launch_mode<5, false>(p, ndim, mode, st);
}

}  // namespace fwi

namespace fwi {

namespace {

// field[slot][node] += w val for every entry of every (slot, tile) bucket, one
// thread per bucket in its entries' order (no two tiles share a node): the
// receiver residuals of one step spread onto an adjoint field.
__global__ void k_inject_buckets(const StepParams p, float* __restrict__ field, int tx, int ty,
                                 int zc, int gx, int gy, int nbuckets) {
  const int bk = blockIdx.x * blockDim.x + threadIdx.x;
  if (bk >= nbuckets) return;
  const int slot = bk / p.ntiles, t = bk - slot * p.ntiles;
  const int bx = t % gx, by = (t / gx) % gy, bz = t / (gx * gy);
  float* f = field + (long long)slot * p.fstride;
  for (int e = p.inj_off[bk]; e < p.inj_off[bk + 1]; ++e) {
    const int loc = p.inj_loc[e];
    const int lx = loc % tx, ly = (loc / tx) % ty, lz = loc / (tx * ty);
    const long long idx = (long long)(bz * zc + lz + p.oz) * p.sxy +
                          (long long)(by * ty + ly + p.oy) * p.sx + (bx * tx + lx + p.ox);
    f[idx] += p.inj_w[e] * p.vals[p.inj_vidx[e] + p.step_off];
  }
}

}  // namespace

cudaError_t launch_inject_buckets(const StepParams& p, float* field, int tx, int ty, int zc, int gx,
                                  int gy, cudaStream_t st) {
  const int n = p.B * p.ntiles;
  if (n <= 0 || !p.inj_off) return cudaSuccess;
  k_inject_buckets<<<(n + 127) / 128, 128, 0, st>>>(p, field, tx, ty, zc, gx, gy, n);
  return cudaGetLastError();
}

}  // namespace fwi
