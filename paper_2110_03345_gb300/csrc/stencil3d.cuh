// Device helpers shared by the TMA-staged 3D kernels (kernels3d_tma.cu,
// kernels3d_x2.cu): the central-difference weights as compile-time constants.
//
// The weights are the unscaled Taylor weights of orders 8 (R = 4) and 10
// (R = 5), second derivative w2[1..R] and first derivative w1[1..R]; with a
// compile-time j they fold into immediate operands of the multiply-adds, so
// the per-axis sums need no constant loads.  The 1/h^2 (1/h) factor of an
// axis is applied once to that axis's sum.
#pragma once

namespace fwi {

template <int R>
__device__ __forceinline__ constexpr float w2c(int j) {
  return R == 4 ? (j == 1 ? 8.0f / 5.0f : j == 2 ? -1.0f / 5.0f : j == 3 ? 8.0f / 315.0f
                                                                         : -1.0f / 560.0f)
                : (j == 1 ? 5.0f / 3.0f : j == 2 ? -5.0f / 21.0f : j == 3 ? 5.0f / 126.0f
                   : j == 4 ? -5.0f / 1008.0f : 1.0f / 3150.0f);
}

template <int R>
__device__ __forceinline__ constexpr float w1c(int j) {
  return R == 4 ? (j == 1 ? 4.0f / 5.0f : j == 2 ? -1.0f / 5.0f : j == 3 ? 4.0f / 105.0f
                                                                         : -1.0f / 280.0f)
                : (j == 1 ? 5.0f / 6.0f : j == 2 ? -5.0f / 21.0f : j == 3 ? 5.0f / 84.0f
                   : j == 4 ? -5.0f / 504.0f : 1.0f / 1260.0f);
}

}  // namespace fwi
