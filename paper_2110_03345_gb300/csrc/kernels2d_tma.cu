// 2D leapfrog step kernels, TMA-staged and looping over shots inside a CTA.
//
// Same arithmetic as kernels2d.cu (damped leapfrog for Eq. 10 of Sec. 2.4,
// exact discrete adjoint, imaging condition of Sec. 2.2 Eq. 8 fused into the
// adjoint), organised for HBM traffic:
//
//  * A CTA owns one 128 x (RY*BY) tile for a group of S shots of the batch.
//    The model fields of the tile (k, and for the variable-density adjoint
//    the b_x / b_y tiles with their halos) are loaded once and reused for the
//    S shots; the adjoint's imaging term sum_s lambda_s h_s is accumulated in
//    registers and added to the group's gradient slot once.  Per shot and
//    grid point the compulsory traffic is then u^n, u^{n-1}, u^{n+1} and h
//    (16 bytes) plus the shared fields divided by S.
//  * Each shot's wavefield tile plus halo (radius R in y, 4 or 8 floats in x)
//    is fetched by one thread with a 3D TMA copy (cp.async.bulk.tensor) into
//    one of two shared-memory buffers, completion tracked by a "full"
//    mbarrier; each warp signals an "empty" mbarrier when it is done with a
//    buffer, and one thread issues the copy for shot k+2 once every warp is
//    done with shot k, while the other warps go on with shot k+1 (no
//    CTA-wide barrier between shots).  Every mbarrier wait is bounded: on
//    time-out the CTA sets an error flag and carries on.
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
};

// One tile (bxi, byi) for shot group grp (shots grp*S .. grp*S+S-1): the body
// shared by the single-problem kernel and the multi-problem kernel.  tmap is
// the tensor map of the wavefield buffer p.u (param or global memory);
// samp_rank is the CTA's rank among its problem's CTAs, gx the problem's tile
// count along x.
template <int R, bool VD, bool ADJ, int RY, int BY>
__device__ __forceinline__ void step2d_tma_tile(const StepParams& p, const AxisW& wx,
                                                const AxisW& wy, const CUtensorMap* tmap,
                                                int bxi, int byi, int gx, int grp,
                                                long long samp_rank, float4* smem, uint64_t* bar) {
  using G = Geo<R, RY, BY>;
  constexpr int TX = G::TX, TY = G::TY, NL = G::NL, SW = G::SW, SH = G::SH, QW = G::QW;
  constexpr int NT = 32 * BY;
  constexpr int NV = 4 + 8 * NL;

  float4* s_t0 = smem;                 // wavefield tile, buffer 0 [SH][SW]
  float4* s_t1 = smem + SH * SW;       // buffer 1
  float4* s_bx = smem + 2 * SH * SW;   // adjoint vd: b_x on tile rows with x halo [TY][SW]
  float4* s_by = s_bx + TY * SW;       // adjoint vd: b_y on tile columns with y halo [SH][QW]

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
  float ay[RY];
#pragma unroll
  for (int iy = 0; iy < RY; ++iy) {
    const int yg = y0 + ty * RY + iy;
    pix[iy] = (yg + p.oy) * p.sx + (xg + p.ox);
    kk[iy] = ldg4(p.kf + pix[iy]);
    ay[iy] = p.spy[yg];
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
  pdl_wait();   // the previous step's wavefields are complete from here on

  if (!ADJ && p.nrec > 0) {
    // receiver sampling of u^n (not written during this step), one thread per slot x receiver
    const long long gid = samp_rank * NT + tid;
    if (gid < (long long)p.B * p.nrec) {
      const int bb = (int)(gid / p.nrec);
      const int r = (int)(gid - (long long)bb * p.nrec);
      const float* ub = p.u + (long long)bb * p.fstride;
      float acc = 0.f;
      for (int c = 0; c < p.ncorner; ++c)
        acc = fmaf(p.smp_w[r * p.ncorner + c], ub[p.smp_node[r * p.ncorner + c]], acc);
      p.smp_out[p.smp_off + (long long)bb * p.nrec + r] = acc;
    }
  }
  if (ns <= 0) return;
  __syncthreads();   // barrier initialisation and the b_x / b_y tiles are visible
  if (tid == 0) {
    mbar_arrive_expect_tx(&bar[0], G::TILE_BYTES);
    tma_load_3d(s_t0, tmap, &bar[0], tmx, tmy, s0);
    if (ns > 1) {
      mbar_arrive_expect_tx(&bar[1], G::TILE_BYTES);
      tma_load_3d(s_t1, tmap, &bar[1], tmx, tmy, s0 + 1);
    }
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
    // latency overlaps it: u^{n-1}, and h^k (adjoint) or b_x, b_y (forward)
    float4 uo[RY], hv[ADJ ? RY : 1];
    float4 bxf[VD && !ADJ ? RY : 1], byf[VD && !ADJ ? RY : 1];
#pragma unroll
    for (int iy = 0; iy < RY; ++iy) {
      uo[iy] = ld4(up_s + pix[iy]);
      if (ADJ && p.image) hv[iy] = __ldcs(reinterpret_cast<const float4*>(h_s + pix[iy]));
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
      float acc[4], c2[4];
#pragma unroll
      for (int ix = 0; ix < 4; ++ix) {
        const int c = 4 * NL + ix;
        c2[ix] = v[c] + v[c];
        float t = 0.f;
#pragma unroll
        for (int j = 1; j <= R; ++j) t = fmaf(wx.w2[j], (v[c + j] + v[c - j]) - c2[ix], t);
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
#pragma unroll
      {
        // y-direction taps on the (x, y) and (z, w) halves of the float4 rows as
        // packed FP32x2 operations: one instruction serves two grid points
        // (round-to-nearest per lane, the same results as the scalar sequence).
        float2 A0 = make_float2(acc[0], acc[1]), A1 = make_float2(acc[2], acc[3]);
        const float2 n0 = make_float2(-c2[0], -c2[1]), n1 = make_float2(-c2[2], -c2[3]);
        float2 D0 = make_float2(0.f, 0.f), D1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          const float4 a = s_u[(srow - j) * SW + tx + NL];
          const float4 c = s_u[(srow + j) * SW + tx + NL];
          const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
          const float2 c0 = make_float2(c.x, c.y), c1 = make_float2(c.z, c.w);
          const float2 w2 = make_float2(wy.w2[j], wy.w2[j]);
          A0 = __ffma2_rn(w2, __fadd2_rn(__fadd2_rn(a0, c0), n0), A0);
          A1 = __ffma2_rn(w2, __fadd2_rn(__fadd2_rn(a1, c1), n1), A1);
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
      }
      if (e1 > e0) {
        // only this row's entries (the bucket's per-row ranges)
        const int* rr = p.inj_row + (size_t)(s * p.ntiles + tile_id) * (TY + 1);
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
      float* upp = up_s + pix[iy];
      const float4 uoi = uo[iy];
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
        gs[iy][0] = fmaf(v[4 * NL + 0], hv[iy].x, gs[iy][0]);
        gs[iy][1] = fmaf(v[4 * NL + 1], hv[iy].y, gs[iy][1]);
        gs[iy][2] = fmaf(v[4 * NL + 2], hv[iy].z, gs[iy][2]);
        gs[iy][3] = fmaf(v[4 * NL + 3], hv[iy].w, gs[iy][3]);
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
      mbar_arrive_expect_tx(&bar[buf], G::TILE_BYTES);
      tma_load_3d(buf ? s_t1 : s_t0, tmap, &bar[buf], tmx, tmy, s + 2);
    }
  }
  if (ADJ && p.image) {
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

template <int R, bool VD, bool ADJ, int RY, int BY>
__global__ void __launch_bounds__(32 * BY, (RY == 1 ? 1024 : 512) / (32 * BY))
k_step2d_tma(const StepParams p, const __grid_constant__ CUtensorMap tmap) {
  pdl_trigger();
  extern __shared__ __align__(128) float4 smem[];
  __shared__ uint64_t bar[4];
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  step2d_tma_tile<R, VD, ADJ, RY, BY>(p, p.wx, p.wy, &tmap, blockIdx.x, blockIdx.y, gridDim.x,
                                      blockIdx.z, blk, smem, bar);
}

// Multi-problem forward step with TMA staging: CTA i advances unit units[i]
// (problem, tile, shot group) by one step; the problem's StepParams and the
// tensor maps of its two wavefield buffers come from descs (global memory).
// UW: every problem of the batch has the same stencil weights (same order and
// spacing), passed as kernel parameters so that the stencil reads them as
// constant operands; otherwise each CTA reads its problem's weights from the
// shared-memory copy of its StepParams.
template <int R, bool VD, int RY, int BY, bool UW>
__global__ void __launch_bounds__(32 * BY, (RY == 1 ? 1024 : 512) / (32 * BY))
k_step2d_tma_multi(const MultiDesc* __restrict__ descs, const MultiUnit* __restrict__ units, int n,
                   const AxisW wx, const AxisW wy) {
  pdl_trigger();
  extern __shared__ __align__(128) float4 smem[];
  __shared__ uint64_t bar[4];
  __shared__ StepParams sp;
  const MultiUnit un = units[blockIdx.x];
  const MultiDesc* d = descs + un.prob;
  {
    const int* src = reinterpret_cast<const int*>(&d->p);
    int* dst = reinterpret_cast<int*>(&sp);
    for (int i = threadIdx.y * 32 + threadIdx.x; i < (int)(sizeof(StepParams) / 4); i += 32 * BY)
      dst[i] = src[i];
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    sp.u = (n & 1) ? d->U1 : d->U0;
    sp.up = (n & 1) ? d->U0 : d->U1;
    sp.step_off = n;
    sp.smp_off = (long long)n * sp.B * sp.nrec;
  }
  __syncthreads();
  const CUtensorMap* map = (n & 1) ? &d->map1 : &d->map0;
  step2d_tma_tile<R, VD, false, RY, BY>(sp, UW ? wx : sp.wx, UW ? wy : sp.wy, map, un.tx, un.ty,
                                        d->gx, un.slot, un.rank, smem, bar);
}

template <int R, bool VD, bool ADJ, int RY, int BY>
constexpr size_t smem_bytes() {
  using G = Geo<R, RY, BY>;
  size_t n = 2 * (size_t)G::SH * G::SW;
  if (VD && ADJ) n += (size_t)G::TY * G::SW + (size_t)G::SH * G::QW;
  return n * sizeof(float4);
}

template <int R, bool VD, bool ADJ, int RY, int BY>
cudaError_t launch_t(const StepParams& p, const CUtensorMap& map, cudaStream_t st) {
  constexpr int TY = RY * BY;
  constexpr size_t smem = smem_bytes<R, VD, ADJ, RY, BY>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_step2d_tma<R, VD, ADJ, RY, BY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_step2d_tma<R, VD, ADJ, RY, BY>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((p.nx + TILE_X - 1) / TILE_X, (p.ny + TY - 1) / TY, (p.B + p.S - 1) / p.S);
  dim3 block(32, BY);
  return launch_pdl(k_step2d_tma<R, VD, ADJ, RY, BY>, grid, block, smem, st, p, map);
}

template <int R, bool VD, bool ADJ>
cudaError_t launch_tile(const StepParams& p, const CUtensorMap& map, int tile, cudaStream_t st) {
  switch (tile) {
    case 1: return launch_t<R, VD, ADJ, 1, 16>(p, map, st);
    case 2: return launch_t<R, VD, ADJ, 2, 16>(p, map, st);
    case 3: return launch_t<R, VD, ADJ, 2, 8>(p, map, st);
    default: return launch_t<R, VD, ADJ, 1, 32>(p, map, st);
  }
}

template <int R, bool VD, int RY, int BY, bool UW>
cudaError_t launch_multi_u(const MultiDesc* descs, const MultiUnit* units, int nunits, int n,
                           const AxisW* w, cudaStream_t st) {
  constexpr size_t smem = smem_bytes<R, VD, false, RY, BY>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_step2d_tma_multi<R, VD, RY, BY, UW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_step2d_tma_multi<R, VD, RY, BY, UW>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (nunits <= 0) return cudaSuccess;
  const AxisW zero{};
  return launch_pdl(k_step2d_tma_multi<R, VD, RY, BY, UW>, dim3(nunits), dim3(32, BY), smem, st,
                    descs, units, n, w ? w[0] : zero, w ? w[1] : zero);
}

template <int R, bool VD, int RY, int BY>
cudaError_t launch_multi_t(const MultiDesc* descs, const MultiUnit* units, int nunits, int n,
                           const AxisW* w, cudaStream_t st) {
  return w ? launch_multi_u<R, VD, RY, BY, true>(descs, units, nunits, n, w, st)
           : launch_multi_u<R, VD, RY, BY, false>(descs, units, nunits, n, w, st);
}

template <int R, bool VD>
cudaError_t launch_multi_tile(const MultiDesc* descs, const MultiUnit* units, int nunits, int n,
                              int tile, const AxisW* w, cudaStream_t st) {
  switch (tile) {
    case 1: return launch_multi_t<R, VD, 1, 16>(descs, units, nunits, n, w, st);
    case 2: return launch_multi_t<R, VD, 2, 16>(descs, units, nunits, n, w, st);
    case 3: return launch_multi_t<R, VD, 2, 8>(descs, units, nunits, n, w, st);
    default: return launch_multi_t<R, VD, 1, 32>(descs, units, nunits, n, w, st);
  }
}

}  // namespace

cudaError_t launch_step2d_tma_multi(const MultiDesc* descs, const MultiUnit* units, int nunits,
                                    int n, int R, bool vd, int tile, const AxisW* w,
                                    cudaStream_t st) {
  if (R == 4) return vd ? launch_multi_tile<4, true>(descs, units, nunits, n, tile, w, st)
                        : launch_multi_tile<4, false>(descs, units, nunits, n, tile, w, st);
  return vd ? launch_multi_tile<5, true>(descs, units, nunits, n, tile, w, st)
            : launch_multi_tile<5, false>(descs, units, nunits, n, tile, w, st);
}

// tile: 0..3, the shapes of tile2_tma_variant
cudaError_t launch_step2d_tma(const StepParams& p, const CUtensorMap& map, int R, bool vd, bool adj,
                              int tile, cudaStream_t st) {
  if (R == 4) {
    if (vd) return adj ? launch_tile<4, true, true>(p, map, tile, st) : launch_tile<4, true, false>(p, map, tile, st);
    return adj ? launch_tile<4, false, true>(p, map, tile, st) : launch_tile<4, false, false>(p, map, tile, st);
  }
  if (vd) return adj ? launch_tile<5, true, true>(p, map, tile, st) : launch_tile<5, true, false>(p, map, tile, st);
  return adj ? launch_tile<5, false, true>(p, map, tile, st) : launch_tile<5, false, false>(p, map, tile, st);
}

// TMA box (floats) of a tile variant: {x extent, y extent}.
void tma_box2d(int R, int tile, int* bx, int* by) {
  const Tile2 t = tile2_tma_variant(tile);
  const int XH = (R <= 4) ? 4 : 8;
  *bx = TILE_X + 2 * XH;
  *by = t.ry * t.by + 2 * R;
}

}  // namespace fwi
