"""GB300-native dense contractions (linalg.matmul, linalg.batch_matmul,
linalg.conv_2d_nhwc_hwcf) behind the C ABI of libnk.so.

Submodules:
  nk     -- ctypes binding of include/nk.h (loads libnk.so; no fallback)
  synth  -- seeded synthetic input generators
  _build -- nvcc build of libnk.so for sm_103a
"""
