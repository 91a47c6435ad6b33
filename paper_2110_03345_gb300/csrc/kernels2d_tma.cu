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
#include "tma2d_tile.cuh"

namespace fwi {

namespace {

template <int R, bool VD, bool ADJ, int RY, int BY, bool CROWD>
__global__ void __launch_bounds__(32 * BY, (RY == 1 ? 1024 : 512) / (32 * BY))
k_step2d_tma(const StepParams p, const __grid_constant__ CUtensorMap tmap,
             const __grid_constant__ CUtensorMap upmap, const __grid_constant__ CUtensorMap hmap) {
  pdl_trigger();
  extern __shared__ __align__(128) float4 smem[];
  __shared__ uint64_t bar[4];
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  step2d_tma_tile<R, VD, ADJ, RY, BY, LEAP, CROWD, true>(p, p.wx, p.wy, &tmap, &upmap, &hmap,
                                                         nullptr, nullptr, blockIdx.x, blockIdx.y,
                                                         gridDim.x, blockIdx.z, blk, smem, bar);
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
  const CUtensorMap* umap = (n & 1) ? &d->imap0 : &d->imap1;   // u^{n-1} = sp.up
  step2d_tma_tile<R, VD, false, RY, BY, LEAP, false, true>(sp, UW ? wx : sp.wx, UW ? wy : sp.wy, map,
                                                           umap, nullptr, nullptr, nullptr, un.tx,
                                                           un.ty, d->gx, un.slot, un.rank, smem,
                                                           bar);
}

template <int R, bool VD, bool ADJ, int RY, int BY, bool CROWD = false>
cudaError_t launch_t(const StepParams& p, const CUtensorMap& map, const CUtensorMap& upmap,
                     const CUtensorMap& hmap, cudaStream_t st) {
  constexpr int TY = RY * BY;
  constexpr size_t smem = smem_bytes<R, VD, ADJ, RY, BY, LEAP, true>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_step2d_tma<R, VD, ADJ, RY, BY, CROWD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_step2d_tma<R, VD, ADJ, RY, BY, CROWD>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((p.nx + TILE_X - 1) / TILE_X, (p.ny + TY - 1) / TY, (p.B + p.S - 1) / p.S);
  dim3 block(32, BY);
  return launch_pdl(k_step2d_tma<R, VD, ADJ, RY, BY, CROWD>, grid, block, smem, st, p, map, upmap,
                    hmap);
}

// the default shape (128 x 16) has a crowded-row instantiation (sinc points)
template <int R, bool VD, bool ADJ>
cudaError_t launch_tile(const StepParams& p, const CUtensorMap& map, const CUtensorMap& um,
                        const CUtensorMap& hm, int tile, cudaStream_t st) {
  switch (tile) {
    case 1:
      return p.inj_crowded ? launch_t<R, VD, ADJ, 1, 16, true>(p, map, um, hm, st)
                           : launch_t<R, VD, ADJ, 1, 16>(p, map, um, hm, st);
    case 2: return launch_t<R, VD, ADJ, 2, 16>(p, map, um, hm, st);
    case 3: return launch_t<R, VD, ADJ, 2, 8>(p, map, um, hm, st);
    default: return launch_t<R, VD, ADJ, 1, 32>(p, map, um, hm, st);
  }
}

template <int R, bool VD, int RY, int BY, bool UW>
cudaError_t launch_multi_u(const MultiDesc* descs, const MultiUnit* units, int nunits, int n,
                           const AxisW* w, cudaStream_t st) {
  constexpr size_t smem = smem_bytes<R, VD, false, RY, BY, LEAP, true>();
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
cudaError_t launch_step2d_tma(const StepParams& p, const CUtensorMap& map, const CUtensorMap& um,
                              const CUtensorMap& hm, int R, bool vd, bool adj, int tile,
                              cudaStream_t st) {
  if (R == 4) {
    if (vd) return adj ? launch_tile<4, true, true>(p, map, um, hm, tile, st)
                       : launch_tile<4, true, false>(p, map, um, hm, tile, st);
    return adj ? launch_tile<4, false, true>(p, map, um, hm, tile, st)
               : launch_tile<4, false, false>(p, map, um, hm, tile, st);
  }
  if (vd) return adj ? launch_tile<5, true, true>(p, map, um, hm, tile, st)
                     : launch_tile<5, true, false>(p, map, um, hm, tile, st);
  return adj ? launch_tile<5, false, true>(p, map, um, hm, tile, st)
             : launch_tile<5, false, false>(p, map, um, hm, tile, st);
}

// TMA box (floats) of a tile variant without halo: {x extent, y extent}.
void tma_box2d_interior(int tile, int* bx, int* by) {
  const Tile2 t = tile2_tma_variant(tile);
  *bx = TILE_X;
  *by = t.ry * t.by;
}

// TMA box (floats) of a tile variant: {x extent, y extent}.
void tma_box2d(int R, int tile, int* bx, int* by) {
  const Tile2 t = tile2_tma_variant(tile);
  const int XH = (R <= 4) ? 4 : 8;
  *bx = TILE_X + 2 * XH;
  *by = t.ry * t.by + 2 * R;
}

}  // namespace fwi
