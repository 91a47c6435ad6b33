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

}  // namespace

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
