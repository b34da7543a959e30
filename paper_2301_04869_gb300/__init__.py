"""GB300-native reduced-space interior-point hot path (arXiv 2301.04869).

Submodules:
  synth  -- seeded synthetic networks and load scenarios (data only)
  ipm    -- ctypes binding of libipm.so (C ABI in include/ipm.h)
  build  -- nvcc build of libipm.so for sm_103a
"""
