"""GB300-native phase-space lattice method for heavy inertial particles (arXiv:1508.02899).

Submodules:
  lat     - binding of the CUDA library (C ABI in include/lat.h); imports fail loudly if the
            library is not built.
  inputs  - seeded synthetic inputs shared by tests and the bench.
  build   - in-tree nvcc build of liblat.so for sm_103a.
"""
