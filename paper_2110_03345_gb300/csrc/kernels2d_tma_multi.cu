// Multi-problem 2D forward step kernels for uneven batches (fwi_batch_*): CTA
// i advances unit units[i] (problem, tile, shot group) by one step with the
// TMA-staged tile body of the single-problem kernels (tma2d_tile.cuh); the
// problem's StepParams and tensor maps come from descs (global memory).
#include "tma2d_tile.cuh"

namespace fwi {

namespace {

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
  return launch_pdl(k_step2d_tma_multi<R, VD, RY, BY, UW>, dim3(nunits), dim3(32, BY), smem,
                    st, descs, units, n, w ? w[0] : zero, w ? w[1] : zero);
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

}  // namespace fwi
