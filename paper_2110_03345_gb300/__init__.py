"""GB300-native acoustic full-waveform-inversion hot path (Stride, arXiv 2110.03345).

Submodules:
  inputs    seeded synthetic phantoms, geometries and wavelets
  binding   ctypes binding of the C ABI (include/fwi.h) over libfwi.so
  build     in-tree nvcc build of libfwi.so for sm_103a
"""
__all__ = ["inputs", "binding", "build"]
