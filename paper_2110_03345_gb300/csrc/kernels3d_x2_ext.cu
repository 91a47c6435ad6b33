// 3D step kernels of the extended schemes of Sec. 2.4 on the two-point
// TMA-staged plane ring of the leapfrog (step3d_x2.cuh): the fourth-order
// time scheme's two passes (EXT_KW, EXT_T4) and the y = 0 attenuation term
// (EXT_ATT0), forward and adjoint, with the arithmetic of kernels_ext.cu.
// The plane ring holds the pass's stencil input (u^n, lambda^k, or the
// k w / k L^T lambda scratch); 64 x 8 columns of 32-plane chunks, one shot
// per CTA.
#include "step3d_x2.cuh"

namespace fwi {

namespace {

constexpr int EXT3_BY = 8;

template <int R, bool VD, bool ADJ, int MODE>
cudaError_t launch_e3(const StepParams& p, const CUtensorMap* const* m, cudaStream_t st) {
  constexpr size_t smem = smem_bytes_x2<R, VD, ADJ, EXT3_BY, MODE>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_step3d_x2<R, VD, ADJ, EXT3_BY, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_step3d_x2<R, VD, ADJ, EXT3_BY, MODE>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((p.nx + 63) / 64, (p.ny + EXT3_BY - 1) / EXT3_BY, p.B * p.nzc);
  return launch_pdl(k_step3d_x2<R, VD, ADJ, EXT3_BY, MODE>, grid, dim3(32, EXT3_BY), smem, st, p,
                    *m[0], *m[1], *m[2], *m[3], *m[4], *m[5], *m[6]);
}

template <int R, bool VD, bool ADJ>
cudaError_t launch_mode3(const StepParams& p, const CUtensorMap* const* m, int mode,
                         cudaStream_t st) {
  switch (mode) {
    case EXT_KW: return launch_e3<R, VD, ADJ, EXT_KW>(p, m, st);
    case EXT_T4: return launch_e3<R, VD, ADJ, EXT_T4>(p, m, st);
    default: return launch_e3<R, VD, ADJ, EXT_ATT0>(p, m, st);
  }
}

}  // namespace

cudaError_t launch_step3d_x2_ext(const StepParams& p, const CUtensorMap& xm, const CUtensorMap& bxm,
                                 const CUtensorMap& bym, const CUtensorMap& upm,
                                 const CUtensorMap& kfm, const CUtensorMap& gm,
                                 const CUtensorMap& hm, int R, bool vd, bool adj, int mode,
                                 cudaStream_t st) {
  if (mode != EXT_KW && mode != EXT_T4 && mode != EXT_ATT0) return cudaErrorInvalidValue;
  const CUtensorMap* m[7] = {&xm, &bxm, &bym, &upm, &kfm, &gm, &hm};
  if (R == 4) {
    if (vd) return adj ? launch_mode3<4, true, true>(p, m, mode, st) : launch_mode3<4, true, false>(p, m, mode, st);
    return adj ? launch_mode3<4, false, true>(p, m, mode, st) : launch_mode3<4, false, false>(p, m, mode, st);
  }
  if (vd) return adj ? launch_mode3<5, true, true>(p, m, mode, st) : launch_mode3<5, true, false>(p, m, mode, st);
  return adj ? launch_mode3<5, false, true>(p, m, mode, st) : launch_mode3<5, false, false>(p, m, mode, st);
}

}  // namespace fwi
