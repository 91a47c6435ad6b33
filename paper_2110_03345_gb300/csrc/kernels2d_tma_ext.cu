// 2D step kernels of the extended schemes of Sec. 2.4 on the TMA-staged
// shot-loop pipeline of the leapfrog (tma2d_tile.cuh): the fourth-order time
// scheme's two passes (EXT_KW, EXT_T4) and the attenuating leapfrog (EXT_ATT0,
// EXT_ATT2), forward and adjoint, with the arithmetic of kernels_ext.cu.
//
// A CTA of 32 x 16 threads owns a 128 x 16 tile for a group of S shots: the
// stencil input x of each shot (u^n, lambda^k, or the k w / k L^T lambda
// scratch of the fourth-order scheme) arrives by a 3D TMA copy, the tile's k
// and attenuation coefficient (and for the y = 2 adjoint the coefficient's
// tiles with halos) are loaded once for the S shots, and the adjoint's
// imaging terms are summed over the S shots in registers and subtracted from
// the group's gradient slot once.
#include "tma2d_tile.cuh"

namespace fwi {

namespace {

constexpr int EXT_BY = 16;   // warps per CTA: one 128-point row per warp

template <int R, bool VD, bool ADJ, int MODE>
__global__ void __launch_bounds__(32 * EXT_BY, 2)
k_step2d_tma_ext(const StepParams p, const __grid_constant__ CUtensorMap tmap,
                 const __grid_constant__ CUtensorMap upmap, const __grid_constant__ CUtensorMap hmap,
                 const __grid_constant__ CUtensorMap h2map,
                 const __grid_constant__ CUtensorMap ucmap) {
  pdl_trigger();
  extern __shared__ __align__(128) float4 smem[];
  __shared__ uint64_t bar[4];
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  step2d_tma_tile<R, VD, ADJ, 1, EXT_BY, MODE, false, true>(p, p.wx, p.wy, &tmap, &upmap, &hmap,
                                                            &h2map, &ucmap, blockIdx.x, blockIdx.y,
                                                            gridDim.x, blockIdx.z, blk, smem, bar);
}

template <int R, bool VD, bool ADJ, int MODE>
cudaError_t launch_e(const StepParams& p, const CUtensorMap* const* maps, cudaStream_t st) {
  constexpr size_t smem = smem_bytes<R, VD, ADJ, 1, EXT_BY, MODE, true>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_step2d_tma_ext<R, VD, ADJ, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_step2d_tma_ext<R, VD, ADJ, MODE>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((p.nx + TILE_X - 1) / TILE_X, (p.ny + EXT_BY - 1) / EXT_BY, (p.B + p.S - 1) / p.S);
  return launch_pdl(k_step2d_tma_ext<R, VD, ADJ, MODE>, grid, dim3(32, EXT_BY), smem, st, p,
                    *maps[0], *maps[1], *maps[2], *maps[3], *maps[4]);
}

template <int R, bool VD, bool ADJ>
cudaError_t launch_mode(const StepParams& p, const CUtensorMap* const* maps, int mode,
                        cudaStream_t st) {
  switch (mode) {
    case EXT_KW: return launch_e<R, VD, ADJ, EXT_KW>(p, maps, st);
    case EXT_T4: return launch_e<R, VD, ADJ, EXT_T4>(p, maps, st);
    case EXT_ATT0: return launch_e<R, VD, ADJ, EXT_ATT0>(p, maps, st);
    default: return launch_e<R, VD, ADJ, EXT_ATT2>(p, maps, st);
  }
}

}  // namespace

// maps: the stencil input p.x with halo, p.up without halo, the history and
// the second history field (4D, step p.hstep; read only by the adjoint when
// p.image), p.u without halo (fourth-order update); tile variant 1 of
// tile2_tma_variant (128 x 16 points).
cudaError_t launch_step2d_tma_ext(const StepParams& p, const CUtensorMap& map,
                                  const CUtensorMap& um, const CUtensorMap& hm,
                                  const CUtensorMap& h2m, const CUtensorMap& ucm, int R, bool vd,
                                  bool adj, int mode, cudaStream_t st) {
  const CUtensorMap* maps[5] = {&map, &um, &hm, &h2m, &ucm};
  if (R == 4) {
    if (vd) return adj ? launch_mode<4, true, true>(p, maps, mode, st) : launch_mode<4, true, false>(p, maps, mode, st);
    return adj ? launch_mode<4, false, true>(p, maps, mode, st) : launch_mode<4, false, false>(p, maps, mode, st);
  }
  if (vd) return adj ? launch_mode<5, true, true>(p, maps, mode, st) : launch_mode<5, true, false>(p, maps, mode, st);
  return adj ? launch_mode<5, false, true>(p, maps, mode, st) : launch_mode<5, false, false>(p, maps, mode, st);
}

}  // namespace fwi
