// 3D leapfrog step kernels, TMA-staged, two x points per thread.
//
// Same arithmetic, in the same order, as the plane-ring kernels of
// kernels3d_tma.cu (Eq. 10 of Sec. 2.4 without attenuation, damped leapfrog,
// exact discrete adjoint, imaging condition of Sec. 2.2 Eq. 8 fused into the
// adjoint), so both give bit-identical results.  What differs is the work
// per instruction:
//
//  * a thread owns two adjacent x points, so a CTA of 32 x BY threads covers
//    a 64 x BY column; every shared-memory read is an 8-byte pair and the
//    arithmetic runs on packed FP32x2 instructions (two lanes, each rounded
//    as the scalar operation);
//  * the z loop advances two planes per trip, so the register queue of the
//    column shifts once per two planes, and one barrier plus one round of
//    TMA refills closes each trip;
//  * the x-y planes (80 floats wide: x0-8 .. x0+71, 16-byte aligned) arrive by
//    4D TMA copies into a ring of R+1+PF planes (the centre, the R planes up
//    to the lead, PF planes in flight); the variable-density adjoint streams
//    b_x on the tile rows and b_y on the tile columns through a second,
//    four-stage ring (two trips), and its per-plane operands (lambda^{k+1},
//    k, h^k, g) through a third, so that no register holds them ahead.
// Every mbarrier wait is bounded: on time-out the error flag is set and the
// kernel carries on, so no thread skips a barrier.
#include "step3d_x2.cuh"

namespace fwi {

namespace {

template <int R, bool VD, bool ADJ, int BY, bool CROWD = false>
cudaError_t launch_t(const StepParams& p, const CUtensorMap& um, const CUtensorMap& bxm,
                     const CUtensorMap& bym, const CUtensorMap* const* om, cudaStream_t st) {
  constexpr size_t smem = smem_bytes_x2<R, VD, ADJ, BY>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_step3d_x2<R, VD, ADJ, BY, X2_LEAP, CROWD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_step3d_x2<R, VD, ADJ, BY, X2_LEAP, CROWD>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((p.nx + 63) / 64, (p.ny + BY - 1) / BY, p.B * p.nzc);
  return launch_pdl(k_step3d_x2<R, VD, ADJ, BY, X2_LEAP, CROWD>, grid, dim3(32, BY), smem, st, p,
                    um, bxm, bym, *om[0], *om[1], *om[2], *om[3]);
}

template <int R, bool VD, bool ADJ>
cudaError_t launch_tile(const StepParams& p, const CUtensorMap& um, const CUtensorMap& bxm,
                        const CUtensorMap& bym, const CUtensorMap* const* om, int tile,
                        cudaStream_t st) {
  // (the 64 x 8 columns of the default variant have a crowded-plane instantiation)
  if (tile3_variant(tile).by == 8)
    return p.inj_crowded ? launch_t<R, VD, ADJ, 8, true>(p, um, bxm, bym, om, st)
                         : launch_t<R, VD, ADJ, 8>(p, um, bxm, bym, om, st);
  return launch_t<R, VD, ADJ, 16>(p, um, bxm, bym, om, st);
}

}  // namespace

cudaError_t launch_step3d_x2(const StepParams& p, const CUtensorMap& um, const CUtensorMap& bxm,
                             const CUtensorMap& bym, const CUtensorMap& upm,
                             const CUtensorMap& kfm, const CUtensorMap& gm,
                             const CUtensorMap& hm, int R, bool vd, bool adj, int tile,
                             cudaStream_t st) {
  const CUtensorMap* om[4] = {&upm, &kfm, &gm, &hm};
  if (R == 4) {
    if (vd) return adj ? launch_tile<4, true, true>(p, um, bxm, bym, om, tile, st)
                       : launch_tile<4, true, false>(p, um, bxm, bym, om, tile, st);
    return adj ? launch_tile<4, false, true>(p, um, bxm, bym, om, tile, st)
               : launch_tile<4, false, false>(p, um, bxm, bym, om, tile, st);
  }
  if (vd) return adj ? launch_tile<5, true, true>(p, um, bxm, bym, om, tile, st)
                     : launch_tile<5, true, false>(p, um, bxm, bym, om, tile, st);
  return adj ? launch_tile<5, false, true>(p, um, bxm, bym, om, tile, st)
             : launch_tile<5, false, false>(p, um, bxm, bym, om, tile, st);
}

}  // namespace fwi
