"""GB300-native acoustic full-waveform-inversion hot path (Stride, arXiv 2110.03345).

Submodules:
  inputs       seeded synthetic phantoms, geometries and wavelets
  binding      ctypes binding of the C ABI (include/fwi.h) over libfwi.so
  build        in-tree nvcc build of libfwi.so for sm_103a
  autograd     torch.autograd.Function of the misfit (backward = adjoint kernel)
  serve        serving loop: requests admitted onto concurrent streams by HBM budget
  autotune     kernel variant and shots-per-CTA tuner (single problems and batches)
  distributed  shot sharding and the gradient sum over ranks
  invert       the inversion loop: frequency blocks, shot subsets, gradient descent
"""
__all__ = ["inputs", "binding", "build", "autograd", "serve", "autotune", "distributed", "invert"]
