"""GB300-native FFT-based homogenization with higher-order terms (arXiv:1712.05145).

Submodules (imported on demand, so that importing the package needs neither a GPU
nor torch):
  build      -- compiles libhom.so (CUDA, sm_103a) in tree
  hom        -- thin ctypes binding of the C ABI in include/hom.h
  synthetic  -- seeded synthetic microstructures (inputs shared with the tests)
"""
__all__ = ["build", "hom", "synthetic"]
