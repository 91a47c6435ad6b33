// The tile body of the TMA-staged 2D step kernels (kernels2d_tma.cu: the
// leapfrog, single- and multi-problem; kernels2d_tma_ext.cu: the extended
// schemes of Sec. 2.4).  One CTA advances one 128 x (RY*BY) tile for a group
// of S shots; each shot's tile plus halo arrives by a 3D TMA copy into one of
// two shared-memory buffers (full / empty mbarriers, bounded waits).
#pragma once

#include "fwi_internal.cuh"
#include "tma_util.cuh"

#include <cuda.h>

namespace fwi {

namespace {

using namespace tma;

__device__ __forceinline__ float4 ldg4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st4(float* p, const float4& v) {
  *reinterpret_cast<float4*>(p) = v;
}
__device__ __forceinline__ float get(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
__device__ __forceinline__ void unpack(const float4& t, float* v) {
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

template <int R, int RY, int BY>
struct Geo {
  static constexpr int TX = TILE_X;
  static constexpr int TY = RY * BY;
  static constexpr int XH = (R <= 4) ? 4 : 8;
  static constexpr int NL = XH / 4;
  static constexpr int SW = TX / 4 + 2 * NL;  // float4 per shared row
  static constexpr int SH = TY + 2 * R;
  static constexpr int QW = TX / 4;
  static constexpr uint32_t TILE_BYTES = (uint32_t)SH * SW * 16;
  // float4 offset of the STG tiles: after the two wavefield buffers and the
  // b_x / b_y (psi) and attenuation (cl) tiles, rounded to 128 bytes
  __host__ __device__ static constexpr int STG_OFF(bool psi, bool cl) {
    return (2 * SH * SW + (psi ? TY * SW + SH * QW : 0) + (cl ? TY * SW + SH * QW : 0) + 7) / 8 * 8;
  }
};

// Update of the float4 of points of one row in an extended scheme (the
// arithmetic of kernels_ext.cu's epilogue): cen = x at the points, acc =
// (L x + injection), lap = its plain Laplacian part (y = 2 forward), lc =
// lap(att lambda) (y = 2 adjoint); the adjoint's imaging terms are added to gs.
constexpr float INV12 = 1.f / 12.f;   // the 1/12 of the fourth-order terms, rounded once

template <bool ADJ, int MODE>
__device__ __forceinline__ void ext_epilogue(const StepParams& p, int s, int pix, int xg, int yg,
                                             const float4& ax4, float ay, const float4& kk,
                                             const float4& at4, const float4& uo4, const float4& uc4,
                                             const float4& h4, const float4* h2s,
                                             const float4* ucs, const float* cen,
                                             const float* acc, const float* lap, const float* lc,
                                             float* gs) {
  const size_t fo = (size_t)s * p.fstride;
  float k[4], ax[4], at[4], uo[4], uc[4], h[4], h2[4], qv[4];
  unpack(kk, k);
  unpack(ax4, ax);
  unpack(at4, at);
  unpack(uo4, uo);
  if (ucs) unpack(*ucs, uc);   // u^n (lambda^k) staged by TMA
  else if (MODE == EXT_T4 && ADJ) unpack(ld4(p.u + fo + pix), uc);
  else unpack(uc4, uc);
  unpack(h4, h);
  if (MODE == EXT_T4 && ADJ && p.image)   // k w^k: staged by TMA (h2s) or read here
    unpack(h2s ? *h2s : __ldcs(reinterpret_cast<const float4*>(p.hist2 + fo + pix)), h2);
  if (MODE == EXT_ATT2) unpack(ld4(p.q + fo + pix), qv);
  bool in[4];
#pragma unroll
  for (int ix = 0; ix < 4; ++ix) in[ix] = (yg < p.ny) && (xg + ix < p.nx);
  float r[4], o1[4], o2[4], qn[4];
#pragma unroll
  for (int ix = 0; ix < 4; ++ix) {
    const float a0 = ax[ix] + ay;
    float rv = 0.f, v1 = 0.f, v2 = 0.f, qq = 0.f;
    if (MODE == EXT_KW) {
      v1 = k[ix] * acc[ix];
    } else if (MODE == EXT_T4) {
      const float F = fmaf(k[ix] * acc[ix], INV12, cen[ix]);
      rv = (2.f * uc[ix] - (1.f - a0) * uo[ix] + F) * __frcp_rn(1.f + a0);
      v1 = F;
      v2 = cen[ix];
      if (ADJ && p.image) gs[ix] = fmaf(cen[ix] * h2[ix], INV12, fmaf(uc[ix], h[ix], gs[ix]));
    } else if (MODE == EXT_ATT0) {
      const float a = a0 + at[ix];
      const float hv = k[ix] * acc[ix];
      rv = (2.f * cen[ix] - (1.f - a) * uo[ix] + hv) * __frcp_rn(1.f + a);
      v1 = hv - 0.5f * at[ix] * (rv - uo[ix]);
      if (ADJ && p.image) gs[ix] = fmaf(cen[ix], h[ix], gs[ix]);
    } else {   // EXT_ATT2
      float E, extra = 0.f;
      if (!ADJ) {
        const float dl = lap[ix] - qv[ix];
        E = fmaf(at[ix], dl, acc[ix]);
        qq = lap[ix];
        extra = 0.5f * k[ix] * at[ix] * dl;
      } else {
        E = acc[ix] + (lc[ix] - qv[ix]);
        qq = lc[ix];
      }
      const float hv = k[ix] * E;
      rv = (2.f * cen[ix] - (1.f - a0) * uo[ix] + hv) * __frcp_rn(1.f + a0);
      v1 = hv + extra;
      if (ADJ && p.image) gs[ix] = fmaf(cen[ix], h[ix], gs[ix]);
    }
    r[ix] = in[ix] ? rv : 0.f;
    o1[ix] = in[ix] ? v1 : 0.f;
    o2[ix] = in[ix] ? v2 : 0.f;
    qn[ix] = in[ix] ? qq : 0.f;
  }
  if (MODE == EXT_KW) {
    st4(p.out + fo + pix, make_float4(o1[0], o1[1], o1[2], o1[3]));
    return;
  }
  st4(p.up + fo + pix, make_float4(r[0], r[1], r[2], r[3]));
  if (MODE == EXT_ATT2) st4(p.q + fo + pix, make_float4(qn[0], qn[1], qn[2], qn[3]));
  if (!ADJ && p.hist) {
    __stcs(reinterpret_cast<float4*>(p.hist + fo + pix), make_float4(o1[0], o1[1], o1[2], o1[3]));
    if (MODE == EXT_T4)
      __stcs(reinterpret_cast<float4*>(p.hist2 + fo + pix), make_float4(o2[0], o2[1], o2[2], o2[3]));
  }
}

// Ask for the lines of a global address in L2 (a hint: no data returns).
__device__ __forceinline__ void prefetch_l2(const void* q) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
}

// One tile (bxi, byi) for shot group grp (shots grp*S .. grp*S+S-1): the body
// shared by the single-problem kernel and the multi-problem kernel.  tmap is
// the tensor map of the wavefield buffer p.u (param or global memory);
// samp_rank is the CTA's rank among its problem's CTAs, gx the problem's tile
// count along x.
// MODE selects the update: LEAP the leapfrog of this file's header, or one
// of the extended schemes (EXT_KW, EXT_T4, EXT_ATT0, EXT_ATT2 of
// fwi_internal.cuh, the arithmetic of kernels_ext.cu) on the same pipeline:
// the stencil input x is the TMA tile (u, lambda, or the k w / k L^T lambda
// scratch of the fourth-order scheme), the model data of the tile (k, the
// attenuation coefficient, its tiles for the y = 2 adjoint) are loaded once
// for the S shots, and the imaging term is summed over the S shots in
// registers.  CROWD: the injection tables have tile rows of more than 32
// entries (sinc points), whose threads find their own entries by bisection
// (a separate instantiation: the unused branch alone cost the leapfrog
// adjoint 2%).  STG: u^{n-1} (upmap, the tile without halo) and, in the
// adjoint, h^k (hmap: (x, y, slot, step), step p.hstep) of each shot arrive
// by TMA with its wavefield tile, two shots ahead, instead of by loads
// that each thread issues before its tile wait.
constexpr int LEAP = -1;

template <int R, bool VD, bool ADJ, int RY, int BY, int MODE = LEAP, bool CROWD = false,
          bool STG = false>
__device__ __forceinline__ void step2d_tma_tile(const StepParams& p, const AxisW& wx,
                                                const AxisW& wy, const CUtensorMap* tmap,
                                                const CUtensorMap* upmap, const CUtensorMap* hmap,
                                                const CUtensorMap* h2map, const CUtensorMap* ucmap,
                                                int bxi, int byi, int gx, int grp,
                                                long long samp_rank, float4* smem, uint64_t* bar) {
  using G = Geo<R, RY, BY>;
  constexpr int TX = G::TX, TY = G::TY, NL = G::NL, SW = G::SW, SH = G::SH, QW = G::QW;
  constexpr int NT = 32 * BY;
  constexpr int NV = 4 + 8 * NL;
  constexpr bool CL = MODE == EXT_ATT2 && ADJ;   // lap(att lambda)
  constexpr bool AT = MODE == EXT_ATT0 || MODE == EXT_ATT2;

  float4* s_t0 = smem;                 // wavefield tile, buffer 0 [SH][SW]
  float4* s_t1 = smem + SH * SW;       // buffer 1
  float4* s_bx = smem + 2 * SH * SW;   // adjoint vd: b_x on tile rows with x halo [TY][SW]
  float4* s_by = s_bx + TY * SW;       // adjoint vd: b_y on tile columns with y halo [SH][QW]
  // y = 2 adjoint: the attenuation coefficient on the tile rows / columns
  float4* s_ax = smem + 2 * SH * SW + ((VD && ADJ) ? TY * SW + SH * QW : 0);
  float4* s_ay = s_ax + TY * SW;
  // STG: u^{n-1}, h^k and (fourth-order adjoint) k w^k tiles [TY][QW] of
  // buffers 0 / 1; the first pass of the fourth-order scheme stages nothing
  constexpr bool SU = STG && MODE != EXT_KW;
  constexpr bool SH2 = SU && MODE == EXT_T4 && ADJ;
  constexpr bool SUC = SU && MODE == EXT_T4;   // u^n (lambda^k) of the fourth-order update
  static_assert(G::STG_OFF(VD && ADJ, CL) % 8 == 0, "TMA destinations on 128-byte boundaries");
  float4* s_uo = smem + G::STG_OFF(VD && ADJ, CL);
  float4* s_hv = s_uo + 2 * TY * QW;
  float4* s_h2 = s_hv + 2 * TY * QW;
  float4* s_uc = s_h2 + 2 * TY * QW;
  constexpr uint32_t IN_BYTES = (uint32_t)TY * QW * 16;   // one tile without halo

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int x0 = bxi * TX, y0 = byi * TY;
  const int s0 = grp * p.S;
  const int ns = min(p.S, p.B - s0);
  const int tile_id = byi * gx + bxi;

  // Model-only set-up first (barriers, sponge, k, the b_x / b_y tiles): in a
  // programmatic dependent launch it overlaps the previous step's tail.
  const int tmx = x0 + p.ox - G::XH;   // multiple of 4 floats: 16-byte aligned box start
  const int tmy = y0 + p.oy - R;
  if (tid == 0) {
    mbar_init(&bar[0], 1);    // full: the TMA copy of a shot's tile landed in buffer 0 / 1
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], BY);   // empty: every warp is done with buffer 0 / 1
    mbar_init(&bar[3], BY);
    fence_mbar_init();
  }
  // Shared model data of the tile, loaded once for the S shots.  Offsets
  // inside one field fit in 32 bits; slot bases are formed once per shot.
  const int xg = x0 + 4 * tx;
  const int base = (y0 + p.oy - R) * p.sx + (x0 + p.ox - G::XH);
  const float4 ax4 = ldg4(p.spx + xg);
  int pix[RY];
  float4 kk[RY];
  float4 atv[AT ? RY : 1];
  float ay[RY];
#pragma unroll
  for (int iy = 0; iy < RY; ++iy) {
    const int yg = y0 + ty * RY + iy;
    pix[iy] = (yg + p.oy) * p.sx + (xg + p.ox);
    kk[iy] = ldg4(p.kf + pix[iy]);
    if (AT) atv[iy] = ldg4(p.att + pix[iy]);
    ay[iy] = p.spy[yg];
  }
  if (ADJ && MODE != EXT_KW && p.image) {
    // the group's gradient slot is read once, after the S shots: its lines
    // are requested in L2 now, so that the read-modify-write at the end hits
    // L2 instead of waiting on DRAM
    const float* gpre = p.g + (size_t)grp * p.fstride;
#pragma unroll
    for (int iy = 0; iy < RY; ++iy) prefetch_l2(gpre + pix[iy]);
  }
  if (VD && ADJ && ns > 0) {
    for (int i = tid; i < TY * SW; i += NT) {
      const int r = i / SW, c = i - r * SW;
      s_bx[i] = ldg4(p.bx + base + (r + R) * p.sx + 4 * c);
    }
    for (int i = tid; i < SH * QW; i += NT) {
      const int r = i / QW, c = i - r * QW;
      s_by[i] = ldg4(p.by + base + r * p.sx + 4 * (c + NL));
    }
  }
  if (CL && ns > 0) {
    for (int i = tid; i < TY * SW; i += NT) {
      const int r = i / SW, c = i - r * SW;
      s_ax[i] = ldg4(p.att + base + (r + R) * p.sx + 4 * c);
    }
    for (int i = tid; i < SH * QW; i += NT) {
      const int r = i / QW, c = i - r * QW;
      s_ay[i] = ldg4(p.att + base + r * p.sx + 4 * (c + NL));
    }
  }
  pdl_wait();   // the previous step's wavefields are complete from here on

  if (!ADJ && p.nrec > 0) {
    // receiver sampling of u^n (not written during this step), a thread or a warp per slot x receiver
    const long long gid = samp_rank * NT + tid;
    sample_receivers(p, gid);
  }
  if (ns <= 0) return;
  __syncthreads();   // barrier initialisation and the b_x / b_y tiles are visible
  // shot k of the group into buffer k & 1: its wavefield tile with halo and,
  // STG, its u^{n-1} and h^k tiles, all on the buffer's full barrier
  const bool stg_h = SU && ADJ && p.image;
  const bool stg_h2 = SH2 && p.image;
  auto issue = [&](int k) {
    const int bf = k & 1;
    mbar_arrive_expect_tx(&bar[bf], G::TILE_BYTES + (SU ? IN_BYTES : 0u) + (stg_h ? IN_BYTES : 0u) +
                                        (stg_h2 ? IN_BYTES : 0u) + (SUC ? IN_BYTES : 0u));
    tma_load_3d(bf ? s_t1 : s_t0, tmap, &bar[bf], tmx, tmy, s0 + k);
    if (SU) {
      tma_load_3d(s_uo + bf * TY * QW, upmap, &bar[bf], x0 + p.ox, y0 + p.oy, s0 + k);
      if (stg_h)   // read once: evict first from L2
        tma_load_4d_hint(s_hv + bf * TY * QW, hmap, &bar[bf], x0 + p.ox, y0 + p.oy, s0 + k, p.hstep,
                         policy_evict_first());
      if (stg_h2)
        tma_load_4d_hint(s_h2 + bf * TY * QW, h2map, &bar[bf], x0 + p.ox, y0 + p.oy, s0 + k, p.hstep,
                         policy_evict_first());
      if (SUC) tma_load_3d(s_uc + bf * TY * QW, ucmap, &bar[bf], x0 + p.ox, y0 + p.oy, s0 + k);
    }
  };
  if (tid == 0) {
    issue(0);
    if (ns > 1) issue(1);
  }
  float gs[RY][4];
#pragma unroll
  for (int iy = 0; iy < RY; ++iy)
#pragma unroll
    for (int q = 0; q < 4; ++q) gs[iy][q] = 0.f;

  for (int k = 0; k < ns; ++k) {
    const int s = s0 + k;
    const int buf = k & 1;
    const float4* s_u = buf ? s_t1 : s_t0;
    float* const up_s = p.up + (size_t)s * p.fstride;
    float* const h_s = p.hist ? p.hist + (size_t)s * p.fstride : nullptr;
    // this shot's global operands are issued before the tile wait, so their
    // latency overlaps it: u^{n-1}, and h^k (adjoint) or b_x, b_y (forward);
    // the extended schemes' u^n (fourth order), k w^k and the Laplacian state
    constexpr bool T4 = MODE == EXT_T4;
    // (the fourth-order adjoint's lambda^k and k w^k and the Laplacian state
    // are read in the update: issued here they would hold registers across
    // the stencil)
    float4 uo[RY], hv[ADJ ? RY : 1], uc[T4 ? RY : 1];   // (STG: unused)
    float4 bxf[VD && !ADJ ? RY : 1], byf[VD && !ADJ ? RY : 1];
#pragma unroll
    for (int iy = 0; iy < RY; ++iy) {
      if (!SU && MODE != EXT_KW) uo[iy] = ld4(up_s + pix[iy]);
      if (!SU && ADJ && MODE != EXT_KW && p.image)
        hv[iy] = __ldcs(reinterpret_cast<const float4*>(h_s + pix[iy]));
      if (T4 && !ADJ && !SUC) uc[iy] = ld4(p.u + (size_t)s * p.fstride + pix[iy]);
      if (VD && !ADJ) {
        bxf[iy] = ldg4(p.bx + pix[iy]);
        byf[iy] = ldg4(p.by + pix[iy]);
      }
    }
    // A wait that times out flags the error and carries on (no early exit, so
    // no thread can miss a later barrier); the host reports FWI_ERR_TIMEOUT.
    if (!mbar_wait_bounded(&bar[buf], (uint32_t)((k >> 1) & 1)) && p.flags) atomicOr(p.flags, 2);
    int e0 = 0, e1 = 0;
    if (p.inj_off) {
      e0 = p.inj_off[s * p.ntiles + tile_id];
      e1 = p.inj_off[s * p.ntiles + tile_id + 1];
    }

#pragma unroll
    for (int iy = 0; iy < RY; ++iy) {
      const int ly = ty * RY + iy;
      const int yg = y0 + ly;
      const int srow = ly + R;
      float v[NV];
#pragma unroll
      for (int q = 0; q <= 2 * NL; ++q) unpack(s_u[srow * SW + tx + q], v + 4 * q);

      // second derivatives in the zero-sum form sum_j w_j (u_{+j} + u_{-j} - 2 u_0)
      // (forward, variable density: the b_x D1x u term is subtracted as soon
      // as D1x u is known, so the four first derivatives are never live at once)
      // y = 2 forward: the plain Laplacian as well (a separate sum only where
      // the b terms of variable density enter acc)
      constexpr bool LAPF = MODE == EXT_ATT2 && !ADJ;
      constexpr bool LAPS = LAPF && VD;
      float acc[4], c2[4], lapx[LAPF ? 4 : 1];
#pragma unroll
      for (int ix = 0; ix < 4; ++ix) {
        const int c = 4 * NL + ix;
        c2[ix] = v[c] + v[c];
        float t = 0.f;
#pragma unroll
        for (int j = 1; j <= R; ++j) t = fmaf(wx.w2[j], (v[c + j] + v[c - j]) - c2[ix], t);
        if (LAPS) lapx[ix] = t;
        if (VD && !ADJ) {
          float d = 0.f;
#pragma unroll
          for (int j = 1; j <= R; ++j) d = fmaf(wx.w1[j], v[c + j] - v[c - j], d);
          t = fmaf(-get(bxf[iy], ix), d, t);
        }
        acc[ix] = t;
      }
      if (VD && ADJ) {
        // D1x(b_x lambda) from the b_x and lambda windows of this row
        float bw[NV];
#pragma unroll
        for (int q = 0; q <= 2 * NL; ++q) unpack(s_bx[ly * SW + tx + q], bw + 4 * q);
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) {
          const int c = 4 * NL + ix;
          float d = 0.f;
#pragma unroll
          for (int j = 1; j <= R; ++j)
            d = fmaf(wx.w1[j], bw[c + j] * v[c + j] - bw[c - j] * v[c - j], d);
          acc[ix] += d;
        }
      }
      {
        // y-direction taps on the (x, y) and (z, w) halves of the float4 rows as
        // packed FP32x2 operations: one instruction serves two grid points
        // (round-to-nearest per lane, the same results as the scalar sequence).
        float2 A0 = make_float2(acc[0], acc[1]), A1 = make_float2(acc[2], acc[3]);
        const float2 n0 = make_float2(-c2[0], -c2[1]), n1 = make_float2(-c2[2], -c2[3]);
        float2 D0 = make_float2(0.f, 0.f), D1 = make_float2(0.f, 0.f);
        float2 P0 = make_float2(0.f, 0.f), P1 = make_float2(0.f, 0.f);   // lap u (LAPS)
        if (LAPS) {
          P0 = make_float2(lapx[0], lapx[1]);
          P1 = make_float2(lapx[2], lapx[3]);
        }
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          const float4 a = s_u[(srow - j) * SW + tx + NL];
          const float4 c = s_u[(srow + j) * SW + tx + NL];
          const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
          const float2 c0 = make_float2(c.x, c.y), c1 = make_float2(c.z, c.w);
          const float2 w2 = make_float2(wy.w2[j], wy.w2[j]);
          A0 = __ffma2_rn(w2, __fadd2_rn(__fadd2_rn(a0, c0), n0), A0);
          A1 = __ffma2_rn(w2, __fadd2_rn(__fadd2_rn(a1, c1), n1), A1);
          if (LAPS) {
            P0 = __ffma2_rn(w2, __fadd2_rn(__fadd2_rn(a0, c0), n0), P0);
            P1 = __ffma2_rn(w2, __fadd2_rn(__fadd2_rn(a1, c1), n1), P1);
          }
          if (VD) {
            const float2 w1 = make_float2(wy.w1[j], wy.w1[j]);
            if (!ADJ) {
              D0 = __ffma2_rn(w1, __fadd2_rn(c0, make_float2(-a0.x, -a0.y)), D0);
              D1 = __ffma2_rn(w1, __fadd2_rn(c1, make_float2(-a1.x, -a1.y)), D1);
            } else {
              // D1y(b_y lambda): b_y(+j) lambda(+j) - b_y(-j) lambda(-j)
              const float4 ba = s_by[(srow - j) * QW + tx];
              const float4 bc = s_by[(srow + j) * QW + tx];
              const float2 t0 = __ffma2_rn(make_float2(-ba.x, -ba.y), a0,
                                           __fmul2_rn(make_float2(bc.x, bc.y), c0));
              const float2 t1 = __ffma2_rn(make_float2(-ba.z, -ba.w), a1,
                                           __fmul2_rn(make_float2(bc.z, bc.w), c1));
              A0 = __ffma2_rn(w1, t0, A0);
              A1 = __ffma2_rn(w1, t1, A1);
            }
          }
        }
        if (VD && !ADJ) {   // - b_y D1y u
          const float4 byv = byf[iy];
          A0 = __ffma2_rn(make_float2(-byv.x, -byv.y), D0, A0);
          A1 = __ffma2_rn(make_float2(-byv.z, -byv.w), D1, A1);
        }
        acc[0] = A0.x; acc[1] = A0.y; acc[2] = A1.x; acc[3] = A1.y;
        if (LAPS) {
          lapx[0] = P0.x; lapx[1] = P0.y; lapx[2] = P1.x; lapx[3] = P1.y;
        } else if (LAPF) {
#pragma unroll
          for (int ix = 0; ix < 4; ++ix) lapx[ix] = acc[ix];
        }
      }
      float lc[CL ? 4 : 1];
      if (CL) {
        // lap(att lambda): the att tiles times the lambda window / column
        float aw[NV];
#pragma unroll
        for (int q = 0; q <= 2 * NL; ++q) unpack(s_ax[ly * SW + tx + q], aw + 4 * q);
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) {
          const int c = 4 * NL + ix;
          const float cc2 = 2.f * (aw[c] * v[c]);
          float t = 0.f;
#pragma unroll
          for (int j = 1; j <= R; ++j)
            t = fmaf(wx.w2[j], (aw[c + j] * v[c + j] + aw[c - j] * v[c - j]) - cc2, t);
          lc[ix] = t;
        }
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          float a[4], c[4], ba[4], bc[4], ac[4];
          unpack(s_u[(srow - j) * SW + tx + NL], a);
          unpack(s_u[(srow + j) * SW + tx + NL], c);
          unpack(s_ay[(srow - j) * QW + tx], ba);
          unpack(s_ay[(srow + j) * QW + tx], bc);
          unpack(s_ay[srow * QW + tx], ac);
#pragma unroll
          for (int ix = 0; ix < 4; ++ix)
            lc[ix] = fmaf(wy.w2[j], (ba[ix] * a[ix] + bc[ix] * c[ix]) - 2.f * (ac[ix] * v[4 * NL + ix]),
                          lc[ix]);
        }
      }
      if (e1 > e0) {
        // only this row's entries (the bucket's per-row ranges)
        const int* rr = p.inj_row + (size_t)(s * p.ntiles + tile_id) * (TY + 1);
        int e = rr[ly], r1 = rr[ly + 1];
        if (CROWD && r1 - e > 32) {
          // a crowded row (sinc points, 8 nodes per point and row): the row's
          // entries sort by position, so this thread's range [e, r1) of
          // positions [lo, lo + 4) comes from two bisections
          const int lo = ly * TX + 4 * tx;
          int a = e, b = r1;
          while (a < b) {
            const int m = (a + b) >> 1;
            if (p.inj_loc[m] < lo) a = m + 1;
            else b = m;
          }
          int c = a;
          b = r1;
          while (c < b) {
            const int m = (c + b) >> 1;
            if (p.inj_loc[m] < lo + 4) c = m + 1;
            else b = m;
          }
          e = a;
          r1 = c;
        }
        for (; e < r1; ++e) {
          const int elx = p.inj_loc[e] - ly * TX;
          if ((elx >> 2) == tx) {
            const float w = (MODE == LEAP) ? p.inj_w[e] : p.inj_scale * p.inj_w[e];
            const float val = w * p.vals[p.inj_vidx[e] + p.step_off];
            const int ix = elx & 3;
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += (q == ix) ? val : 0.f;
          }
        }
      }
      if (MODE != LEAP) {
        const int so = buf * TY * QW + ly * QW + tx;   // this thread's float4 in a staged tile
        const float4 uoe = SU ? s_uo[so] : uo[iy];
        const float4 hve = (SU && ADJ && MODE != EXT_KW) ? s_hv[so]
                           : ((ADJ && MODE != EXT_KW) ? hv[iy] : uo[iy]);
        ext_epilogue<ADJ, MODE>(p, s, pix[iy], xg, yg, ax4, ay[iy], kk[iy],
                                AT ? atv[iy] : make_float4(0.f, 0.f, 0.f, 0.f), uoe,
                                T4 ? uc[iy] : uo[iy], hve, SH2 ? s_h2 + so : nullptr,
                                SUC ? s_uc + so : nullptr, v + 4 * NL,
                                acc, LAPF ? lapx : acc, CL ? lc : acc, gs[iy]);
        continue;
      }
      float* upp = up_s + pix[iy];
      const float4 uoi = SU ? s_uo[buf * TY * QW + ly * QW + tx] : uo[iy];
      float res[4], upd[4];
#pragma unroll
      for (int ix = 0; ix < 4; ++ix) {
        const float a = get(ax4, ix) + ay[iy];
        const float h = get(kk[iy], ix) * acc[ix];
        const float cen = v[4 * NL + ix];
        const float r = (2.f * cen - (1.f - a) * get(uoi, ix) + h) * __frcp_rn(1.f + a);
        const bool in = (yg < p.ny) && (xg + ix < p.nx);
        res[ix] = in ? r : 0.f;
        upd[ix] = in ? h : 0.f;
      }
      st4(upp, make_float4(res[0], res[1], res[2], res[3]));
      if (!ADJ) {
        if (h_s)
          __stcs(reinterpret_cast<float4*>(h_s + pix[iy]),
                 make_float4(upd[0], upd[1], upd[2], upd[3]));
      } else if (p.image) {
        const float4 hvi = SU ? s_hv[buf * TY * QW + ly * QW + tx] : hv[iy];
        gs[iy][0] = fmaf(v[4 * NL + 0], hvi.x, gs[iy][0]);
        gs[iy][1] = fmaf(v[4 * NL + 1], hvi.y, gs[iy][1]);
        gs[iy][2] = fmaf(v[4 * NL + 2], hvi.z, gs[iy][2]);
        gs[iy][3] = fmaf(v[4 * NL + 3], hvi.w, gs[iy][3]);
      }
    }
    // This warp is done with the buffer.  Thread 0 refills it for shot k + 2
    // once every warp has arrived; the other warps go on to shot k + 1 (its
    // tile is already loading), so no CTA-wide barrier separates the shots.
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(&bar[2 + buf]);
    if (tid == 0 && k + 2 < ns) {
      if (!mbar_wait_bounded(&bar[2 + buf], (uint32_t)((k >> 1) & 1)) && p.flags)
        atomicOr(p.flags, 2);
      fence_proxy_async_smem();
      issue(k + 2);
    }
  }
  if (ADJ && MODE != EXT_KW && p.image) {
    // g_group -= sum over this group's shots of lambda^k h^k
    float* gbase = p.g + (size_t)grp * p.fstride;
#pragma unroll
    for (int iy = 0; iy < RY; ++iy) {
      float* gp = gbase + pix[iy];
      float4 g = ld4(gp);
      g.x -= gs[iy][0];
      g.y -= gs[iy][1];
      g.z -= gs[iy][2];
      g.w -= gs[iy][3];
      st4(gp, g);
    }
  }
}

// Dynamic shared memory of the tile body: two wavefield buffers, the b_x /
// b_y tiles of the variable-density adjoint, the attenuation tiles of the
// y = 2 adjoint.
template <int R, bool VD, bool ADJ, int RY, int BY, int MODE = LEAP, bool STG = false>
constexpr size_t smem_bytes() {
  using G = Geo<R, RY, BY>;
  size_t n = G::STG_OFF(VD && ADJ, MODE == EXT_ATT2 && ADJ);
  // u^{n-1} (and h^k, and the fourth-order adjoint's k w^k) tiles, two buffers
  // (fourth order: u^{n-1}, h^k, k w^k and u^n slots in both directions)
  if (STG && MODE != EXT_KW)
    n += (size_t)(MODE == EXT_T4 ? 8 : (ADJ ? 4 : 2)) * G::TY * G::QW;
  return n * sizeof(float4);
}

}  // namespace

}  // namespace fwi
