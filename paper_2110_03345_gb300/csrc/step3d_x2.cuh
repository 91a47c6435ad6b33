// The two-point TMA-staged 3D step kernel (kernels3d_x2.cu: the leapfrog;
// kernels3d_x2_ext.cu: the fourth-order time scheme's passes and the y = 0
// attenuation term of Sec. 2.4 on the same plane ring).
#pragma once

#include "fwi_internal.cuh"
#include "stencil3d.cuh"
#include "tma_util.cuh"

#include <cuda.h>

namespace fwi {

namespace {


using namespace tma;

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 lds2(const float* p) {
  return *reinterpret_cast<const float2*>(p);
}

template <int R, int BY, bool PSI = false>
struct GeoX2 {
  static constexpr int TXP = 64;            // x points of a CTA row (32 threads x 2)
  static constexpr int BXW = 80;            // floats per staged row: x0-8 .. x0+71
  static constexpr int XOFF = 8;            // column of x0 in a staged row
  static constexpr int BYH = BY + 2 * R;    // staged rows: y0-R .. y0+BY+R-1
  static constexpr int PLANE = BYH * BXW;   // floats per staged plane (a multiple of 32)
  // planes in flight ahead of the lead (the variable-density adjoint keeps
  // two: with its b stages the ring then takes 73 KB of shared memory)
  static constexpr int PF = PSI ? 2 : 3;
  static constexpr int NSU = R + 1 + PF;    // ring depth
  static constexpr int M = (R + 1) / 2;     // x pairs on each side of the own pair
  static constexpr uint32_t PLANE_BYTES = PLANE * 4;
  // variable-density adjoint: a b stage holds b_x on the tile rows (80 x BY,
  // x0-8 .. x0+71) and b_y on the tile columns (64 x BYH, x0 .. x0+63)
  static constexpr int BXB = BXW * BY;
  static constexpr int BYB = TXP * BYH;
  static constexpr int BSTAGE = BXB + BYB;
  static constexpr uint32_t BSTAGE_BYTES = BSTAGE * 4;
  // variable-density adjoint: a stage of per-plane operands holds the
  // column's lambda^{k+1}, k, h^k and g tiles (64 x BY each)
  static constexpr int OPT = TXP * BY;
  static constexpr int NOS = 4;             // operand stages: two loop trips
};

// MODE: X2_LEAP the leapfrog, or EXT_KW / EXT_T4 / EXT_ATT0 (fwi_internal.cuh)
// with the arithmetic of kernels_ext.cu: the plane ring holds the stencil
// input (u^n, lambda^k, or the k w / k L^T lambda scratch), and the update
// writes k (L x + s) (EXT_KW) or the fourth-order / attenuating update.
constexpr int X2_LEAP = -1;
constexpr float X2_INV12 = 1.f / 12.f;   // the fourth-order scheme's 1/12, rounded once

// CROWD: the injection tables have planes of more than 32 entries in a tile
// (the 64-node rows of sinc points), whose threads find their own pair's
// entries by bisection (a separate instantiation).
template <int R, bool VD, bool ADJ, int BY, int MODE = X2_LEAP, bool CROWD = false>
__global__ void __launch_bounds__(32 * BY, ((VD && ADJ) ? 512 : 768) / (32 * BY))
k_step3d_x2(const StepParams p, const __grid_constant__ CUtensorMap umap,
            const __grid_constant__ CUtensorMap bxmap, const __grid_constant__ CUtensorMap bymap,
            const __grid_constant__ CUtensorMap opup, const __grid_constant__ CUtensorMap opkf,
            const __grid_constant__ CUtensorMap opg, const __grid_constant__ CUtensorMap oph) {
  pdl_trigger();
  using G = GeoX2<R, BY, VD && ADJ>;
  constexpr int TY = BY;
  constexpr int NT = 32 * BY;
  constexpr int Q = 2 * R + 1;
  constexpr int NSU = G::NSU;
  constexpr int M = G::M;
  constexpr int BXW = G::BXW;
  constexpr bool PSI = VD && ADJ;
  extern __shared__ __align__(128) float smem3x[];
  float* ring = smem3x;                       // [NSU][BYH][BXW]
  constexpr int NBS = 4;                      // b stages: two loop trips of two planes
  float* bring = ring + NSU * G::PLANE;       // PSI: [NBS stages][b_x [BY][BXW], b_y [BYH][TXP]]
  constexpr int NOS = G::NOS;
  // operand stages (variable density): [NOS][lambda^{k+1}, k, h, g][BY][TXP]
  // in the adjoint, [NOS][u^{n-1}, k][BY][TXP] in the forward
  constexpr bool OPS = VD;
  constexpr int OPN = ADJ ? 4 : 2;            // operand tiles per stage
  float* ops = bring + (PSI ? NBS * G::BSTAGE : 0);
  __shared__ uint64_t bar[NSU];
  __shared__ uint64_t bbar[NBS];
  __shared__ uint64_t obar[NOS];
  __shared__ int s_pe[MAX_ZCHUNK + 1];        // first source entry of each plane of the chunk

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int b = blockIdx.z / p.nzc;
  const int zc = blockIdx.z - b * p.nzc;
  const int x0 = blockIdx.x * G::TXP, y0 = blockIdx.y * TY;
  const int z0 = zc * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.nz);
  const int nz_c = z1 - z0;
  const int nplanes = nz_c + 2 * R;
  const size_t fo = (size_t)b * p.fstride;
  const int xg = x0 + 2 * tx, yg = y0 + ty;
  const long long col = (long long)(yg + p.oy) * p.sx + (xg + p.ox);   // even: 8-byte pairs


  const int tmx = x0 + p.ox - G::XOFF;      // 16-byte aligned box start
  const int tmy = y0 + p.oy - R;
  const int pz0 = z0 - R + p.oz;            // padded z of staged plane 0
  if (tid == 0) {
    for (int k = 0; k < NSU; ++k) mbar_init(&bar[k], 1);
    for (int k = 0; k < NBS; ++k) mbar_init(&bbar[k], 1);
    for (int k = 0; k < NOS; ++k) mbar_init(&obar[k], 1);
    fence_mbar_init();
  }
  // Source entries of the tile are sorted by tile-local index, which grows
  // with the plane: s_pe[lz] = first entry of plane lz (binary search), so a
  // plane's entries are s_pe[lz] .. s_pe[lz + 1] - 1.
  bool has_inj = false;
  if (p.inj_off) {
    const int t = b * p.ntiles + (zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int e0 = p.inj_off[t], e1 = p.inj_off[t + 1];
    has_inj = e1 > e0;
    if (has_inj) {
      for (int k = tid; k <= nz_c; k += NT) {
        const int lim = k * (TY * G::TXP);
        int lo = e0, hi = e1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (__ldg(p.inj_loc + mid) < lim) lo = mid + 1;
          else hi = mid;
        }
        s_pe[k] = lo;
      }
    }
  }
  pdl_wait();   // the previous step's wavefields are complete from here on
  if (!ADJ && p.nrec > 0) {
    // receiver sampling of u^n (not written during this step), a thread or a warp per slot x receiver
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const long long gid = blk * NT + tid;
    sample_receivers(p, gid);
  }
  if (nz_c <= 0) return;
  __syncthreads();
  // OPS: the operands of plane ii of the chunk into operand stage ii % NOS
  const bool img = ADJ && p.image;
  auto issue_ops = [&](int ii) {
    const int st = ii % NOS;
    float* o = ops + st * OPN * G::OPT;
    const int xx = x0 + p.ox, yy = y0 + p.oy, zz = z0 + ii + p.oz;
    mbar_arrive_expect_tx(&obar[st], (uint32_t)G::OPT * 4u * (img ? 4u : 2u));
    tma_load_4d(o, &opup, &obar[st], xx, yy, zz, b);
    tma_load_4d(o + G::OPT, &opkf, &obar[st], xx, yy, zz, 0);
    if (img) {   // h^k is read once: evict first from L2
      tma_load_5d_hint(o + 2 * G::OPT, &oph, &obar[st], xx, yy, zz, b, p.hstep,
                       policy_evict_first());
      tma_load_4d(o + 3 * G::OPT, &opg, &obar[st], xx, yy, zz, b);
    }
  };
  if (tid == 0) {
    if (OPS)
      for (int ii = 0; ii < NOS && ii < nz_c; ++ii) issue_ops(ii);
    for (int lp = 0; lp < NSU && lp < nplanes; ++lp) {
      mbar_arrive_expect_tx(&bar[lp], G::PLANE_BYTES);
      tma_load_4d(ring + lp * G::PLANE, &umap, &bar[lp], tmx, tmy, pz0 + lp, b);
    }
    if (PSI) {
      for (int i = 0; i < NBS && i < nz_c; ++i) {
        float* st = bring + i * G::BSTAGE;
        mbar_arrive_expect_tx(&bbar[i], G::BSTAGE_BYTES);
        tma_load_4d(st, &bxmap, &bbar[i], tmx, y0 + p.oy, z0 + i + p.oz, 0);
        tma_load_4d(st + G::BXB, &bymap, &bbar[i], x0 + p.ox, tmy, z0 + i + p.oz, 0);
      }
    }
  }

  const int c0 = G::XOFF + 2 * tx;          // own pair's column in a staged row (even)
  const int own = (ty + R) * BXW + c0;
  bool timed_out = false;
  // register queues, U planes per loop trip: q[j] = u at plane z0 + i0 - R + j
  // of this column (i0 = first plane of the trip); shifted by U after a trip
  constexpr int U = 2;
  float2 q[Q + U - 1];
  float2 qz[PSI ? Q + U - 1 : 1];
  // planes 0 .. R-1 (halo only)
#pragma unroll
  for (int lp = 0; lp < R; ++lp) {
    if (!mbar_wait_bounded(&bar[lp], 0)) timed_out = true;
    q[lp] = lds2(ring + lp * G::PLANE + own);
    if (PSI)
      qz[lp] = __fmul2_rn(__ldg(reinterpret_cast<const float2*>(p.bz + (long long)(pz0 + lp) * p.sxy + col)),
                          q[lp]);
  }
  __syncthreads();   // their slots take planes NSU .. NSU+R-1
  if (tid == 0) {
    for (int lp = NSU; lp < NSU + R && lp < nplanes; ++lp) {
      const int k = lp % NSU;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar[k], G::PLANE_BYTES);
      tma_load_4d(ring + k * G::PLANE, &umap, &bar[k], tmx, tmy, pz0 + lp, b);
    }
  }
  // planes R .. 2R-1
#pragma unroll
  for (int lp = R; lp < 2 * R; ++lp) {
    if (!mbar_wait_bounded(&bar[lp % NSU], (uint32_t)((lp / NSU) & 1))) timed_out = true;
    q[lp] = lds2(ring + (lp % NSU) * G::PLANE + own);
    if (PSI)
      qz[lp] = __fmul2_rn(__ldg(reinterpret_cast<const float2*>(p.bz + (long long)(pz0 + lp) * p.sxy + col)),
                          q[lp]);
  }

  const float ay = p.spy[yg];
  const float2 axy = make_float2(p.spx[xg] + ay, p.spx[xg + 1] + ay);
  const bool in_y = yg < p.ny;
  const bool in0 = in_y && xg < p.nx, in1 = in_y && xg + 1 < p.nx;

  const int loc0 = ty * G::TXP + 2 * tx;    // entry location of the own pair in plane lz = 0

  constexpr bool KWM = MODE == EXT_KW, T4M = MODE == EXT_T4, A0M = MODE == EXT_ATT0;
  // (the extended schemes' u^n (lambda^k), k w^k and damping: x[0..2], only
  // in their instantiations)
  constexpr int NX = (MODE == X2_LEAP) ? 1 : 3;
  struct Ops {
    float2 uo, kk, hv, gv, bx, by, bz, bzl;
    float2 x[NX];
    float sz;   // sponge damping of the plane (z part)
  };
  auto ldg2 = [](const float* a) { return __ldg(reinterpret_cast<const float2*>(a)); };
  auto load_ops = [&](int ii) {
    const float2 z2 = make_float2(0.f, 0.f);
    Ops o;
    o.uo = o.kk = o.hv = o.gv = o.bx = o.by = o.bz = o.bzl = z2;
#pragma unroll
    for (int q = 0; q < NX; ++q) o.x[q] = z2;
    o.sz = __ldg(p.spz + z0 + ii);
    const long long id = (long long)(z0 + ii + p.oz) * p.sxy + col;
    if (T4M) {
      o.x[0] = *reinterpret_cast<const float2*>(p.u + fo + id);
      if (ADJ && p.image) o.x[1] = __ldcs(reinterpret_cast<const float2*>(p.hist2 + fo + id));
    }
    if (A0M) o.x[2] = ldg2(p.att + id);
    if (PSI) {   // lambda^{k+1}, k, h, g come from the operand stages
      o.bzl = ldg2(p.bz + (long long)(pz0 + ii + 2 * R) * p.sxy + col);
      return o;
    }
    if (!OPS) {   // (OPS: u^{n-1} and k come from the operand stages)
      o.uo = *reinterpret_cast<const float2*>(p.up + fo + id);
      o.kk = ldg2(p.kf + id);
    }
    if (ADJ && p.image) {
      o.hv = __ldcs(reinterpret_cast<const float2*>(p.hist + fo + id));
      o.gv = *reinterpret_cast<const float2*>(p.g + fo + id);
    }
    if (VD && !ADJ) {
      o.bx = ldg2(p.bx + id);
      o.by = ldg2(p.by + id);
      o.bz = ldg2(p.bz + id);
    }
    if (PSI) o.bzl = ldg2(p.bz + (long long)(pz0 + ii + 2 * R) * p.sxy + col);
    return o;
  };
  Ops nxt = load_ops(0);

  for (int i0 = 0; i0 < nz_c; i0 += U) {
#pragma unroll
    for (int s = 0; s < U; ++s) {
      const int i = i0 + s;
      if (i < nz_c) {
        const int z = z0 + i;
        const long long idx = (long long)(z + p.oz) * p.sxy + col;
        const Ops cur = nxt;
        if (i + 1 < nz_c) nxt = load_ops(i + 1);
        // the lead plane z + R completes the queue
        const int lead = i + 2 * R;
        const int sl = lead % NSU;
        if (!mbar_wait_bounded(&bar[sl], (uint32_t)((lead / NSU) & 1))) timed_out = true;
        q[s + 2 * R] = lds2(ring + sl * G::PLANE + own);
        if (PSI) qz[s + 2 * R] = __fmul2_rn(cur.bzl, q[s + 2 * R]);
        const float* cp = ring + ((i + R) % NSU) * G::PLANE;   // centre plane z
        const float* bxp = bring + (i % NBS) * G::BSTAGE;   // b_x rows of the tile
        const float* byp = bxp + G::BXB;                    // b_y columns with the y halo
        if (PSI && !mbar_wait_bounded(&bbar[i % NBS], (uint32_t)((i / NBS) & 1))) timed_out = true;

        // x pairs of the centre row: columns c0 - 2M .. c0 + 2M + 1
        float2 X[2 * M + 1];
#pragma unroll
        for (int k = 0; k <= 2 * M; ++k) X[k] = lds2(cp + (ty + R) * BXW + c0 - 2 * M + 2 * k);
        auto ux = [&](int d) {   // u at column c0 + d
          const int e = d + 2 * M;
          return (e & 1) ? X[e >> 1].y : X[e >> 1].x;
        };
        float2 Yp[R + 1], Ym[R + 1];
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          Yp[j] = lds2(cp + (ty + R + j) * BXW + c0);
          Ym[j] = lds2(cp + (ty + R - j) * BXW + c0);
        }

        // zero-sum second derivatives per axis, sum_j w_j (u_{+j} + u_{-j} - 2 u_0),
        // with the unscaled weights as immediates; 1/h^2 applied per axis
        const float2 cen = q[s + R];
        const float2 n2 = make_float2(-(cen.x + cen.x), -(cen.y + cen.y));
        const float2 z2 = make_float2(0.f, 0.f);
        float2 ax = z2, ay = z2, az = z2;
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          const float2 xp = make_float2(ux(j), ux(j + 1));
          const float2 xm = make_float2(ux(-j), ux(1 - j));
          ax = __ffma2_rn(bc2(w2c<R>(j)), __fadd2_rn(__fadd2_rn(xp, xm), n2), ax);
          ay = __ffma2_rn(bc2(w2c<R>(j)), __fadd2_rn(__fadd2_rn(Yp[j], Ym[j]), n2), ay);
          az = __ffma2_rn(bc2(w2c<R>(j)),
                          __fadd2_rn(__fadd2_rn(q[s + R + j], q[s + R - j]), n2), az);
        }
        float2 acc = __fmul2_rn(ax, bc2(p.ih2[0]));
        acc = __ffma2_rn(ay, bc2(p.ih2[1]), acc);
        acc = __ffma2_rn(az, bc2(p.ih2[2]), acc);
        if (VD && !ADJ) {
          float2 dx = z2, dy = z2, dz = z2;
#pragma unroll
          for (int j = 1; j <= R; ++j) {
            const float2 xp = make_float2(ux(j), ux(j + 1));
            const float2 xm = make_float2(ux(-j), ux(1 - j));
            dx = __ffma2_rn(bc2(w1c<R>(j)), __fadd2_rn(xp, neg2(xm)), dx);
            dy = __ffma2_rn(bc2(w1c<R>(j)), __fadd2_rn(Yp[j], neg2(Ym[j])), dy);
            dz = __ffma2_rn(bc2(w1c<R>(j)),
                            __fadd2_rn(q[s + R + j], neg2(q[s + R - j])), dz);
          }
          float2 t = __fmul2_rn(cur.bx, __fmul2_rn(dx, bc2(p.ih1[0])));
          t = __ffma2_rn(cur.by, __fmul2_rn(dy, bc2(p.ih1[1])), t);
          t = __ffma2_rn(cur.bz, __fmul2_rn(dz, bc2(p.ih1[2])), t);
          acc = __fadd2_rn(acc, neg2(t));
        }
        if (PSI) {
          // b_x lambda on the centre row, b_y lambda on the centre column
          float2 PX[2 * M + 1];
#pragma unroll
          for (int k = 0; k <= 2 * M; ++k)
            PX[k] = __fmul2_rn(lds2(bxp + ty * BXW + c0 - 2 * M + 2 * k), X[k]);
          auto px = [&](int d) {
            const int e = d + 2 * M;
            return (e & 1) ? PX[e >> 1].y : PX[e >> 1].x;
          };
          float2 sx = z2, sy = z2, sz = z2;
#pragma unroll
          for (int j = 1; j <= R; ++j) {
            const float2 pp = make_float2(px(j), px(j + 1));
            const float2 pm = make_float2(px(-j), px(1 - j));
            sx = __ffma2_rn(bc2(w1c<R>(j)), __fadd2_rn(pp, neg2(pm)), sx);
            const float2 yb = __fmul2_rn(lds2(byp + (ty + R + j) * G::TXP + c0 - G::XOFF), Yp[j]);
            const float2 ya = __fmul2_rn(lds2(byp + (ty + R - j) * G::TXP + c0 - G::XOFF), Ym[j]);
            sy = __ffma2_rn(bc2(w1c<R>(j)), __fadd2_rn(yb, neg2(ya)), sy);
            sz = __ffma2_rn(bc2(w1c<R>(j)),
                            __fadd2_rn(qz[s + R + j], neg2(qz[s + R - j])), sz);
          }
          acc = __ffma2_rn(sx, bc2(p.ih1[0]), acc);
          acc = __ffma2_rn(sy, bc2(p.ih1[1]), acc);
          acc = __ffma2_rn(sz, bc2(p.ih1[2]), acc);
        }
        if (has_inj) {
          const int lz = z - z0;
          const int l0 = lz * (TY * G::TXP) + loc0;
          int e = s_pe[lz], pe1 = s_pe[lz + 1];
          if (CROWD && pe1 - e > 32) {
            // entries sort by position: this pair's [l0, l0 + 2) by two bisections
            int a = e, bnd = pe1;
            while (a < bnd) {
              const int m = (a + bnd) >> 1;
              if (__ldg(p.inj_loc + m) < l0) a = m + 1;
              else bnd = m;
            }
            int c = a;
            bnd = pe1;
            while (c < bnd) {
              const int m = (c + bnd) >> 1;
              if (__ldg(p.inj_loc + m) < l0 + 2) c = m + 1;
              else bnd = m;
            }
            e = a;
            pe1 = c;
          }
          if constexpr (CROWD) {
            for (; e < pe1; ++e) {
              const int l = __ldg(p.inj_loc + e);
              const float w = (MODE == X2_LEAP) ? p.inj_w[e] : p.inj_scale * p.inj_w[e];
              if (l == l0) acc.x = fmaf(w, p.vals[p.inj_vidx[e] + p.step_off], acc.x);
              else if (l == l0 + 1) acc.y = fmaf(w, p.vals[p.inj_vidx[e] + p.step_off], acc.y);
            }
          } else {
            const int pe1c = s_pe[lz + 1];
            for (int e2 = s_pe[lz]; e2 < pe1c; ++e2) {
              const int l = __ldg(p.inj_loc + e2);
              if (l == l0)
                acc.x = fmaf(MODE == X2_LEAP ? p.inj_w[e2] : p.inj_scale * p.inj_w[e2],
                             p.vals[p.inj_vidx[e2] + p.step_off], acc.x);
              else if (l == l0 + 1)
                acc.y = fmaf(MODE == X2_LEAP ? p.inj_w[e2] : p.inj_scale * p.inj_w[e2],
                             p.vals[p.inj_vidx[e2] + p.step_off], acc.y);
            }
          }
        }
        float2 uo = cur.uo, kk = cur.kk, hv = cur.hv, gv = cur.gv;
        if (OPS) {   // this plane's operand stage
          if (!mbar_wait_bounded(&obar[i % NOS], (uint32_t)((i / NOS) & 1))) timed_out = true;
          const float* o = ops + (i % NOS) * OPN * G::OPT + ty * G::TXP + 2 * tx;
          uo = lds2(o);
          kk = lds2(o + G::OPT);
          if (img) {
            hv = lds2(o + 2 * G::OPT);
            gv = lds2(o + 3 * G::OPT);
          }
        }
        const float sz_ = cur.sz;
        const float2 a = make_float2(axy.x + sz_, axy.y + sz_);
        if constexpr (MODE != X2_LEAP) {
          // the extended schemes' update, lane by lane (kernels_ext.cu's arithmetic)
          const float cn[2] = {cen.x, cen.y}, ac[2] = {acc.x, acc.y}, kv[2] = {kk.x, kk.y};
          const float2 uc2 = cur.x[0], h22 = cur.x[NX > 1 ? 1 : 0], at2 = cur.x[NX > 2 ? 2 : 0];
          const float uov[2] = {uo.x, uo.y}, ucv[2] = {uc2.x, uc2.y};
          const float hvv[2] = {hv.x, hv.y}, h2v[2] = {h22.x, h22.y};
          const float gvv[2] = {gv.x, gv.y}, atv[2] = {at2.x, at2.y};
          const float av[2] = {a.x, a.y};
          const bool inl[2] = {in0, in1};
#pragma unroll
          for (int l = 0; l < 2; ++l) {
            if (!inl[l]) continue;
            const long long o = fo + idx + l;
            if (KWM) {
              p.out[o] = kv[l] * ac[l];
              continue;
            }
            float r, hval = 0.f;
            if (T4M) {
              const float F = fmaf(kv[l] * ac[l], X2_INV12, cn[l]);
              r = (2.f * ucv[l] - (1.f - av[l]) * uov[l] + F) * __frcp_rn(1.f + av[l]);
              hval = F;
            } else {   // A0M
              const float aa = av[l] + atv[l];
              const float hh = kv[l] * ac[l];
              r = (2.f * cn[l] - (1.f - aa) * uov[l] + hh) * __frcp_rn(1.f + aa);
              hval = hh - 0.5f * atv[l] * (r - uov[l]);
            }
            p.up[o] = r;
            if (!ADJ) {
              if (p.hist) {
                __stcs(p.hist + o, hval);
                if (T4M) __stcs(p.hist2 + o, cn[l]);
              }
            } else if (p.image) {
              p.g[o] = T4M ? gvv[l] - fmaf(cn[l] * h2v[l], X2_INV12, ucv[l] * hvv[l])
                           : fmaf(-cn[l], hvv[l], gvv[l]);
            }
          }
          continue;
        }
        const float2 h = __fmul2_rn(kk, acc);
        float2 t = __ffma2_rn(make_float2(-(1.f - a.x), -(1.f - a.y)), uo,
                              make_float2(2.f * cen.x, 2.f * cen.y));
        t = __fadd2_rn(t, h);
        const float2 r = __fmul2_rn(t, make_float2(__frcp_rn(1.f + a.x), __frcp_rn(1.f + a.y)));
        if (in1) {
          *reinterpret_cast<float2*>(p.up + fo + idx) = r;
          if (!ADJ) {
            if (p.hist) __stcs(reinterpret_cast<float2*>(p.hist + fo + idx), h);
          } else if (p.image) {
            *reinterpret_cast<float2*>(p.g + fo + idx) = __ffma2_rn(neg2(cen), hv, gv);
          }
        } else if (in0) {
          p.up[fo + idx] = r.x;
          if (!ADJ) {
            if (p.hist) __stcs(p.hist + fo + idx, h.x);
          } else if (p.image) {
            p.g[fo + idx] = fmaf(-cen.x, hv.x, gv.x);
          }
        }
      }
    }
    // one barrier per loop trip: every thread is done with the trip's centre
    // planes and b stages, whose slots take the planes R + NSU and NBS ahead
    __syncthreads();
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < U; ++s) {
        const int i = i0 + s;
        if (i < nz_c) {
          const int nx_ = i + R + NSU;   // the centre plane's slot takes plane nx_
          if (nx_ < nplanes) {
            const int k = nx_ % NSU;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[k], G::PLANE_BYTES);
            tma_load_4d(ring + k * G::PLANE, &umap, &bar[k], tmx, tmy, pz0 + nx_, b);
          }
          if (OPS && i + NOS < nz_c) {   // the stage of plane i takes plane i + NOS
            fence_proxy_async_smem();
            issue_ops(i + NOS);
          }
          if (PSI && i + NBS < nz_c) {
            const int st = i % NBS;
            const int zb = z0 + i + NBS + p.oz;
            float* sb = bring + st * G::BSTAGE;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bbar[st], G::BSTAGE_BYTES);
            tma_load_4d(sb, &bxmap, &bbar[st], tmx, y0 + p.oy, zb, 0);
            tma_load_4d(sb + G::BXB, &bymap, &bbar[st], x0 + p.ox, tmy, zb, 0);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < Q - 1; ++j) {
      q[j] = q[j + U];
      if (PSI) qz[j] = qz[j + U];
    }
  }
  if (timed_out && p.flags) atomicOr(p.flags, 2);
}

template <int R, bool VD, bool ADJ, int BY, int MODE = X2_LEAP>
constexpr size_t smem_bytes_x2() {
  using G = GeoX2<R, BY, VD && ADJ>;
  size_t n = (size_t)G::NSU * G::PLANE;
  if (VD && ADJ) n += 4 * (size_t)G::BSTAGE + (size_t)G::NOS * 4 * G::OPT;   // b and operand stages
  if (VD && !ADJ) n += (size_t)G::NOS * 2 * G::OPT;                         // operand stages
  return n * sizeof(float);
}

}  // namespace

}  // namespace fwi
