"""GB300-native hybrid Fourier / real-space Gaussian-mixture galaxy x PSF
renderer (Lang 2020, arXiv:2012.15797).

  build      compiles the CUDA library (lib/libmogconv.so) for sm_103a
  capi       ctypes binding of include/mogconv.h (same names)
  renderer   torch-tensor marshalling around the C-ABI (Renderer)

Importing ``capi`` or ``renderer`` requires the built library and raises
otherwise; there is no CPU fallback.
"""

__all__ = ["build", "capi", "renderer"]
