// 3D leapfrog step kernels (forward and adjoint) for sm_103a: 2.5D blocking.
//
// Same scheme as the 2D kernels (Eq. 10 of Sec. 2.4 without attenuation,
// damped leapfrog, exact discrete adjoint with the imaging condition of
// Sec. 2.2 Eq. 8 fused into the adjoint step).
//
// A CTA of 32 x BY threads owns a 32 x BY column of one shot and streams
// along z over a chunk of planes.  Each thread keeps the 2R+1 values of its
// own column (z-R .. z+R) in a register queue, so z derivatives never touch
// shared memory; the current x-y plane is staged in shared memory from the
// queue centre, with only the x/y halo loaded from global memory (L2).  In
// the variable-density adjoint, b_z * lambda is kept in a second queue and
// b_x * lambda, b_y * lambda are staged as plane tiles.
#include "fwi_internal.cuh"

namespace fwi {

namespace {

template <int R, bool VD, bool ADJ, int BY>
__global__ void __launch_bounds__(32 * BY)
k_step3d(const StepParams p) {
  constexpr int TX = 32, TY = BY;
  constexpr int SW = TX + 2 * R, SH = TY + 2 * R;
  constexpr int NT = 32 * BY;
  constexpr int Q = 2 * R + 1;
  constexpr bool PSI = VD && ADJ;
  __shared__ float s_u[SH][SW];
  __shared__ float s_px[PSI ? TY : 1][PSI ? SW : 1];
  __shared__ float s_py[PSI ? SH : 1][PSI ? TX : 1];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int b = blockIdx.z / p.nzc;
  const int zc = blockIdx.z - b * p.nzc;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = zc * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.nz);
  const long long fo = (long long)b * p.fstride;
  const float* __restrict__ u = p.u + fo;
  const int xg = x0 + tx, yg = y0 + ty;
  const long long col = (long long)(yg + p.oy) * p.sx + (xg + p.ox);

  if (!ADJ && p.nrec > 0) {
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const long long gid = blk * NT + tid;
    sample_receivers(p, gid);
  }

  // Register queues: q[j] = u at plane z - R + j of this thread's column.
  float q[Q];
  float qz[PSI ? Q : 1];
#pragma unroll
  for (int j = 0; j < Q - 1; ++j) {
    const long long o = col + (long long)(z0 - R + j + p.oz) * p.sxy;
    q[j] = u[o];
    if (PSI) qz[j] = p.bz[o] * q[j];
  }

  const float axy = p.spx[xg] + p.spy[yg];
  const bool in_xy = (xg < p.nx) && (yg < p.ny);
  int e0 = 0, e1 = 0;
  if (p.inj_off) {
    const int t = b * p.ntiles + (zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    e0 = p.inj_off[t];
    e1 = p.inj_off[t + 1];
  }
  const int nTop = R * SW;

  for (int z = z0; z < z1; ++z) {
    const long long pz = (long long)(z + p.oz) * p.sxy;
    {
      const long long o = col + pz + (long long)R * p.sxy;
      q[Q - 1] = u[o];
      if (PSI) qz[Q - 1] = p.bz[o] * q[Q - 1];
    }
    __syncthreads();   // previous plane's readers are done with the shared tiles
    const long long pb = pz + (long long)(y0 + p.oy - R) * p.sx + (x0 + p.ox - R);
    for (int i = tid; i < 2 * nTop + TY * 2 * R; i += NT) {
      int r, c;
      if (i < nTop) {
        r = i / SW; c = i - r * SW;
      } else if (i < 2 * nTop) {
        const int k = i - nTop;
        r = R + TY + k / SW; c = k % SW;
      } else {
        const int k = i - 2 * nTop;
        r = R + k / (2 * R);
        const int cc = k % (2 * R);
        c = cc < R ? cc : TX + cc;
      }
      s_u[r][c] = u[pb + (long long)r * p.sx + c];
    }
    s_u[ty + R][tx + R] = q[R];
    if (PSI) {
      // psi_x on the tile rows with x halo, psi_y on the tile columns with y halo
      for (int i = tid; i < TY * SW; i += NT) {
        const int r = i / SW, c = i - r * SW;
        const long long o = pb + (long long)(r + R) * p.sx + c;
        s_px[r][c] = p.bx[o] * u[o];
      }
      for (int i = tid; i < SH * TX; i += NT) {
        const int r = i / TX, c = i - r * TX;
        const long long o = pb + (long long)r * p.sx + c + R;
        s_py[r][c] = p.by[o] * u[o];
      }
    }
    __syncthreads();

    // zero-sum form sum_j w_j (u_{+j} + u_{-j} - 2 u_0): exact 0 on constants
    const float cen = q[R];
    const float c2 = cen + cen;
    float acc = 0.f;
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      acc = fmaf(p.wx.w2[j], (s_u[ty + R][tx + R + j] + s_u[ty + R][tx + R - j]) - c2, acc);
      acc = fmaf(p.wy.w2[j], (s_u[ty + R + j][tx + R] + s_u[ty + R - j][tx + R]) - c2, acc);
      acc = fmaf(p.wz.w2[j], (q[R + j] + q[R - j]) - c2, acc);
    }
    const long long idx = col + pz;
    if (VD && !ADJ) {
      float dx = 0.f, dy = 0.f, dz = 0.f;
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        dx = fmaf(p.wx.w1[j], s_u[ty + R][tx + R + j] - s_u[ty + R][tx + R - j], dx);
        dy = fmaf(p.wy.w1[j], s_u[ty + R + j][tx + R] - s_u[ty + R - j][tx + R], dy);
        dz = fmaf(p.wz.w1[j], q[R + j] - q[R - j], dz);
      }
      acc -= __ldg(p.bx + idx) * dx + __ldg(p.by + idx) * dy + __ldg(p.bz + idx) * dz;
    }
    if (PSI) {
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        acc = fmaf(p.wx.w1[j], s_px[ty][tx + R + j] - s_px[ty][tx + R - j], acc);
        acc = fmaf(p.wy.w1[j], s_py[ty + R + j][tx] - s_py[ty + R - j][tx], acc);
        acc = fmaf(p.wz.w1[j], qz[R + j] - qz[R - j], acc);
      }
    }
    if (e1 > e0) {
      const int lz = z - z0;
      for (int e = e0; e < e1; ++e) {
        const int loc = p.inj_loc[e];
        if (loc == (lz * TY + ty) * TX + tx)
          acc += p.inj_w[e] * p.vals[p.inj_vidx[e] + p.step_off];
      }
    }

    const float a = axy + p.spz[z];
    const float h = __ldg(p.kf + idx) * acc;
    float* upp = p.up + fo + idx;
    const float r = (2.f * cen - (1.f - a) * (*upp) + h) * __frcp_rn(1.f + a);
    if (in_xy) {
      *upp = r;
      if (!ADJ) {
        if (p.hist) __stcs(p.hist + fo + idx, h);
      } else if (p.image) {
        float* gp = p.g + fo + idx;
        *gp = fmaf(-cen, __ldcs(p.hist + fo + idx), *gp);
      }
    }
#pragma unroll
    for (int j = 0; j < Q - 1; ++j) {
      q[j] = q[j + 1];
      if (PSI) qz[j] = qz[j + 1];
    }
  }
}

template <int R, bool VD, bool ADJ, int BY>
cudaError_t launch_t(const StepParams& p, cudaStream_t st) {
  dim3 grid((p.nx + 31) / 32, (p.ny + BY - 1) / BY, p.B * p.nzc);
  dim3 block(32, BY);
  k_step3d<R, VD, ADJ, BY><<<grid, block, 0, st>>>(p);
  return cudaGetLastError();
}

template <int R, bool VD, bool ADJ>
cudaError_t launch_tile(const StepParams& p, int tile, cudaStream_t st) {
  return tile3_variant(tile).by == 8 ? launch_t<R, VD, ADJ, 8>(p, st)
                                     : launch_t<R, VD, ADJ, 16>(p, st);
}

}  // namespace

cudaError_t launch_step3d(const StepParams& p, int R, bool vd, bool adj, int tile,
                          cudaStream_t st) {
  if (R == 4) {
    if (vd) return adj ? launch_tile<4, true, true>(p, tile, st) : launch_tile<4, true, false>(p, tile, st);
    return adj ? launch_tile<4, false, true>(p, tile, st) : launch_tile<4, false, false>(p, tile, st);
  }
  if (vd) return adj ? launch_tile<5, true, true>(p, tile, st) : launch_tile<5, true, false>(p, tile, st);
  return adj ? launch_tile<5, false, true>(p, tile, st) : launch_tile<5, false, false>(p, tile, st);
}

size_t step3d_smem(int R, bool vd, bool adj, int tile) {
  const int by = tile3_variant(tile).by;
  const int SW = 32 + 2 * R, SH = by + 2 * R;
  size_t n = (size_t)SH * SW;
  if (vd && adj) n += (size_t)by * SW + (size_t)SH * 32;
  return n * sizeof(float);
}

}  // namespace fwi
