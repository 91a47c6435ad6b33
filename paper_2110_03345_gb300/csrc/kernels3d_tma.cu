// 3D leapfrog step kernels, TMA-staged (2.5D blocking with a plane ring).
//
// Same scheme as kernels3d.cu (Eq. 10 of Sec. 2.4 without attenuation,
// damped leapfrog, exact discrete adjoint, imaging condition of Sec. 2.2
// Eq. 8 fused into the adjoint), in the explicit rounding order shared with
// the two-point kernels of kernels3d_x2.cu (bit-identical results).  A CTA
// of 32 x BY threads owns a 32 x BY column of one shot and streams along z
// over a chunk of planes:
//
//  * each x-y plane of the column, with its halo, arrives by a 4D TMA copy
//    (x, y, z, shot) into a ring of 2R+2 shared-memory planes, so the copies
//    of the next planes run while the current plane is computed;
//  * a thread keeps the 2R+1 values of its own column in a register queue,
//    filled from the ring as each plane arrives (z derivatives in registers),
//    and reads the x / y neighbours of the centre plane from the ring;
//  * the variable-density adjoint also needs b_x, b_y with their halos on the
//    centre plane: they come through a second, two-stage TMA ring; b_z
//    lambda is queued like lambda.
// Every mbarrier wait is bounded (on time-out the error flag is set and the
// kernel carries on, so no thread skips a barrier).
#include "fwi_internal.cuh"
#include "stencil3d.cuh"
#include "tma_util.cuh"

#include <cuda.h>

namespace fwi {

namespace {

using namespace tma;

template <int R, int BY>
struct Geo3 {
  static constexpr int BXW = 48;             // floats per staged row: x0-8 .. x0+39
  static constexpr int XOFF = 8;             // column of x0 in a staged row
  static constexpr int BYH = BY + 2 * R;     // staged rows: y0-R .. y0+BY+R-1
  static constexpr int PLANE = BYH * BXW;    // floats per staged plane
  static constexpr int NSU = 2 * R + 2;      // ring depth (centre .. lead + 1 prefetch)
  static constexpr uint32_t PLANE_BYTES = PLANE * 4;
};

template <int R, bool VD, bool ADJ, int BY>
__global__ void __launch_bounds__(32 * BY, 1024 / (32 * BY))
k_step3d_tma(const StepParams p, const __grid_constant__ CUtensorMap umap,
             const __grid_constant__ CUtensorMap bxmap, const __grid_constant__ CUtensorMap bymap) {
  pdl_trigger();
  using G = Geo3<R, BY>;
  constexpr int TX = 32, TY = BY;
  constexpr int NT = 32 * BY;
  constexpr int Q = 2 * R + 1;
  constexpr bool PSI = VD && ADJ;
  constexpr int NSU = G::NSU;
  extern __shared__ __align__(128) float smem3[];
  float* ring = smem3;                       // [NSU][BYH][BXW]
  float* bring = ring + NSU * G::PLANE;      // PSI: [2 stages][b_x, b_y][BYH][BXW]
  __shared__ uint64_t bar[NSU];
  __shared__ uint64_t bbar[2];
  __shared__ int s_pe[MAX_ZCHUNK + 1];        // first source entry of each plane of the chunk

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int b = blockIdx.z / p.nzc;
  const int zc = blockIdx.z - b * p.nzc;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = zc * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.nz);
  const int nz_c = z1 - z0;
  const int nplanes = nz_c + 2 * R;
  const size_t fo = (size_t)b * p.fstride;
  const int xg = x0 + tx, yg = y0 + ty;
  const long long col = (long long)(yg + p.oy) * p.sx + (xg + p.ox);


  const int tmx = x0 + p.ox - G::XOFF;     // 16-byte aligned box start
  const int tmy = y0 + p.oy - R;
  const int pz0 = z0 - R + p.oz;           // padded z of staged plane 0
  if (tid == 0) {
    for (int k = 0; k < NSU; ++k) mbar_init(&bar[k], 1);
    mbar_init(&bbar[0], 1);
    mbar_init(&bbar[1], 1);
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
        const int lim = k * (TY * TX);
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
  // receiver sampling of u^n (not written during this step), a thread or a warp per slot x receiver
  if (!ADJ && p.nrec > 0) {
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const long long gid = blk * NT + tid;
    sample_receivers(p, gid);
  }
  if (nz_c <= 0) return;
  __syncthreads();
  if (tid == 0) {
    for (int lp = 0; lp < NSU && lp < nplanes; ++lp) {
      mbar_arrive_expect_tx(&bar[lp], G::PLANE_BYTES);
      tma_load_4d(ring + lp * G::PLANE, &umap, &bar[lp], tmx, tmy, pz0 + lp, b);
    }
    if (PSI) {
      for (int i = 0; i < 2 && i < nz_c; ++i) {
        mbar_arrive_expect_tx(&bbar[i], 2 * G::PLANE_BYTES);
        tma_load_4d(bring + (2 * i) * G::PLANE, &bxmap, &bbar[i], tmx, tmy, z0 + i + p.oz, 0);
        tma_load_4d(bring + (2 * i + 1) * G::PLANE, &bymap, &bbar[i], tmx, tmy, z0 + i + p.oz, 0);
      }
    }
  }

  const int own = (ty + R) * G::BXW + tx + G::XOFF;   // own column in a staged plane
  bool timed_out = false;
  // register queues, U planes per loop trip: q[j] = u at plane z0 + i0 - R + j
  // of this column (i0 = first plane of the trip); shifted by U after a trip
  constexpr int U = 2;
  float q[Q + U - 1];
  float qz[PSI ? Q + U - 1 : 1];
#pragma unroll
  for (int lp = 0; lp < Q - 1; ++lp) {
    if (!mbar_wait_bounded(&bar[lp], 0)) timed_out = true;
    q[lp] = ring[lp * G::PLANE + own];
    if (PSI) qz[lp] = __fmul_rn(__ldg(p.bz + (long long)(pz0 + lp) * p.sxy + col), q[lp]);
  }
  __syncthreads();   // planes 0..R-1 are halo-only: their buffers take planes NSU..NSU+R-1
  if (tid == 0) {
    for (int lp = NSU; lp < NSU + R && lp < nplanes; ++lp) {
      const int k = lp % NSU;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar[k], G::PLANE_BYTES);
      tma_load_4d(ring + k * G::PLANE, &umap, &bar[k], tmx, tmy, pz0 + lp, b);
    }
  }

  const float axy = p.spx[xg] + p.spy[yg];
  const bool in_xy = (xg < p.nx) && (yg < p.ny);

  const int r0 = ty + R, c0 = tx + G::XOFF;

  // Global operands of a point (u^{n-1}, k, h, g, b) are loaded one plane
  // ahead (software pipelining in registers), so their latency overlaps a plane.
  struct Ops {
    float uo, kk, hv, gv, bx, by, bz, bzl;
    float sz;   // sponge damping of the plane (z part)
  };
  auto load_ops = [&](int ii) {
    Ops o{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    o.sz = __ldg(p.spz + z0 + ii);
    const long long id = (long long)(z0 + ii + p.oz) * p.sxy + col;
    o.uo = p.up[fo + id];
    o.kk = __ldg(p.kf + id);
    if (ADJ && p.image) {
      o.hv = __ldcs(p.hist + fo + id);
      o.gv = p.g[fo + id];
    }
    if (VD && !ADJ) {
      o.bx = __ldg(p.bx + id);
      o.by = __ldg(p.by + id);
      o.bz = __ldg(p.bz + id);
    }
    if (PSI) o.bzl = __ldg(p.bz + (long long)(pz0 + ii + 2 * R) * p.sxy + col);
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
        const float uo = cur.uo, kk = cur.kk, hv = cur.hv, bxv = cur.bx, byv = cur.by,
                    bzv = cur.bz;
        // the lead plane z + R completes the queue
        const int lead = i + 2 * R;
        if (!mbar_wait_bounded(&bar[lead % NSU], (uint32_t)((lead / NSU) & 1))) timed_out = true;
        q[s + 2 * R] = ring[(lead % NSU) * G::PLANE + own];
        if (PSI) qz[s + 2 * R] = __fmul_rn(cur.bzl, q[s + 2 * R]);
        const float* cp = ring + ((i + R) % NSU) * G::PLANE;   // centre plane z
        const float* bxp = bring + (2 * (i & 1)) * G::PLANE;
        const float* byp = bxp + G::PLANE;
        if (PSI && !mbar_wait_bounded(&bbar[i & 1], (uint32_t)((i >> 1) & 1))) timed_out = true;

        // zero-sum second derivatives per axis, sum_j w_j (u_{+j} + u_{-j} - 2 u_0),
        // with the unscaled weights as immediates; 1/h^2 applied per axis
        const float cen = q[s + R];
        const float n2 = -(cen + cen);
        float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          ax = fmaf(w2c<R>(j), (cp[r0 * G::BXW + c0 + j] + cp[r0 * G::BXW + c0 - j]) + n2, ax);
          ay = fmaf(w2c<R>(j), (cp[(r0 + j) * G::BXW + c0] + cp[(r0 - j) * G::BXW + c0]) + n2, ay);
          az = fmaf(w2c<R>(j), (q[s + R + j] + q[s + R - j]) + n2, az);
        }
        float acc = __fmul_rn(ax, p.ih2[0]);
        acc = fmaf(ay, p.ih2[1], acc);
        acc = fmaf(az, p.ih2[2], acc);
        if (VD && !ADJ) {
          float dx = 0.f, dy = 0.f, dz = 0.f;
#pragma unroll
          for (int j = 1; j <= R; ++j) {
            dx = fmaf(w1c<R>(j), cp[r0 * G::BXW + c0 + j] + (-cp[r0 * G::BXW + c0 - j]), dx);
            dy = fmaf(w1c<R>(j), cp[(r0 + j) * G::BXW + c0] + (-cp[(r0 - j) * G::BXW + c0]), dy);
            dz = fmaf(w1c<R>(j), q[s + R + j] + (-q[s + R - j]), dz);
          }
          float t = __fmul_rn(bxv, __fmul_rn(dx, p.ih1[0]));
          t = fmaf(byv, __fmul_rn(dy, p.ih1[1]), t);
          t = fmaf(bzv, __fmul_rn(dz, p.ih1[2]), t);
          acc = acc + (-t);
        }
        if (PSI) {
          float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
          for (int j = 1; j <= R; ++j) {
            const int xp = r0 * G::BXW + c0 + j, xm = r0 * G::BXW + c0 - j;
            const int yp = (r0 + j) * G::BXW + c0, ym = (r0 - j) * G::BXW + c0;
            sx = fmaf(w1c<R>(j), __fmul_rn(bxp[xp], cp[xp]) + (-__fmul_rn(bxp[xm], cp[xm])), sx);
            sy = fmaf(w1c<R>(j), __fmul_rn(byp[yp], cp[yp]) + (-__fmul_rn(byp[ym], cp[ym])), sy);
            sz = fmaf(w1c<R>(j), qz[s + R + j] + (-qz[s + R - j]), sz);
          }
          acc = fmaf(sx, p.ih1[0], acc);
          acc = fmaf(sy, p.ih1[1], acc);
          acc = fmaf(sz, p.ih1[2], acc);
        }
        if (has_inj) {
          const int lz = z - z0;
          const int me = (lz * TY + ty) * TX + tx;
          const int pe1 = s_pe[lz + 1];
          for (int e = s_pe[lz]; e < pe1; ++e)
            if (__ldg(p.inj_loc + e) == me)
              acc = fmaf(p.inj_w[e], p.vals[p.inj_vidx[e] + p.step_off], acc);
        }
        const float a = axy + cur.sz;
        // explicit rounding order (no contraction left to the compiler), shared
        // with the two-point kernels of kernels3d_x2.cu
        const float h = __fmul_rn(kk, acc);
        float t = fmaf(-(1.f - a), uo, 2.f * cen);
        t = __fadd_rn(t, h);
        const float r = __fmul_rn(t, __frcp_rn(1.f + a));
        if (in_xy) {
          p.up[fo + idx] = r;
          if (!ADJ) {
            if (p.hist) __stcs(p.hist + fo + idx, h);
          } else if (p.image) {
            p.g[fo + idx] = fmaf(-cen, hv, cur.gv);
          }
        }
        __syncthreads();   // every thread is done with the centre plane and this b stage
        if (tid == 0) {
          const int nxp = i + R + NSU;   // the centre plane's buffer takes plane nxp
          if (nxp < nplanes) {
            const int k = nxp % NSU;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[k], G::PLANE_BYTES);
            tma_load_4d(ring + k * G::PLANE, &umap, &bar[k], tmx, tmy, pz0 + nxp, b);
          }
          if (PSI && i + 2 < nz_c) {
            const int st = i & 1;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bbar[st], 2 * G::PLANE_BYTES);
            tma_load_4d(bring + (2 * st) * G::PLANE, &bxmap, &bbar[st], tmx, tmy, z + 2 + p.oz, 0);
            tma_load_4d(bring + (2 * st + 1) * G::PLANE, &bymap, &bbar[st], tmx, tmy,
                        z + 2 + p.oz, 0);
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

template <int R, bool VD, bool ADJ, int BY>
constexpr size_t smem_bytes3() {
  using G = Geo3<R, BY>;
  size_t n = (size_t)G::NSU * G::PLANE;
  if (VD && ADJ) n += 4 * (size_t)G::PLANE;
  return n * sizeof(float);
}

template <int R, bool VD, bool ADJ, int BY>
cudaError_t launch_t(const StepParams& p, const CUtensorMap& um, const CUtensorMap& bxm,
                     const CUtensorMap& bym, cudaStream_t st) {
  constexpr size_t smem = smem_bytes3<R, VD, ADJ, BY>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_step3d_tma<R, VD, ADJ, BY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_step3d_tma<R, VD, ADJ, BY>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((p.nx + 31) / 32, (p.ny + BY - 1) / BY, p.B * p.nzc);
  return launch_pdl(k_step3d_tma<R, VD, ADJ, BY>, grid, dim3(32, BY), smem, st, p, um, bxm, bym);
}

template <int R, bool VD, bool ADJ>
cudaError_t launch_tile(const StepParams& p, const CUtensorMap& um, const CUtensorMap& bxm,
                        const CUtensorMap& bym, int tile, cudaStream_t st) {
  return tile3_variant(tile).by == 8 ? launch_t<R, VD, ADJ, 8>(p, um, bxm, bym, st)
                                     : launch_t<R, VD, ADJ, 16>(p, um, bxm, bym, st);
}

}  // namespace

cudaError_t launch_step3d_tma(const StepParams& p, const CUtensorMap& um, const CUtensorMap& bxm,
                              const CUtensorMap& bym, int R, bool vd, bool adj, int tile,
                              cudaStream_t st) {
  if (R == 4) {
    if (vd) return adj ? launch_tile<4, true, true>(p, um, bxm, bym, tile, st)
                       : launch_tile<4, true, false>(p, um, bxm, bym, tile, st);
    return adj ? launch_tile<4, false, true>(p, um, bxm, bym, tile, st)
               : launch_tile<4, false, false>(p, um, bxm, bym, tile, st);
  }
  if (vd) return adj ? launch_tile<5, true, true>(p, um, bxm, bym, tile, st)
                     : launch_tile<5, true, false>(p, um, bxm, bym, tile, st);
  return adj ? launch_tile<5, false, true>(p, um, bxm, bym, tile, st)
             : launch_tile<5, false, false>(p, um, bxm, bym, tile, st);
}

// TMA box rows (y extent) of a 3D tile variant.
int tma_box3d_rows(int R, int tile) { return tile3_variant(tile).by + 2 * R; }

}  // namespace fwi
