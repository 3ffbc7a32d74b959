"""GB300-native iPiano solver for the FoE despeckling model (Chen et al.,
"A higher-order MRF based variational model for multiplicative noise
reduction").

Submodules:
  synth - seeded synthetic inputs (images, speckle, filter bank)
  fe    - the binding to the CUDA library libfe.so (C ABI in include/fe.h);
          importing it loads the library and raises if it is missing
"""
__all__ = ["synth", "fe"]
