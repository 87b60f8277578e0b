"""GB300 (sm_103a) implementation of the Neural Bounding hot path (Liu et al., SIGGRAPH 2024).

Submodules:
  inputs  seeded synthetic scenes, queries and initial weights (no method arithmetic)
  nb      ctypes binding of libnb (include/nb.h); the compute runs in libnb's CUDA kernels
  build   in-tree nvcc build of libnb.so
"""
