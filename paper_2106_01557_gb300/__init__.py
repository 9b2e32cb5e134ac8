"""GB300-native (sm_103a) implementation of the fused f+g time step of the
thermal liquid-vapor lattice Boltzmann model of Huang, Wu & Adams (PRL 2021).

Submodules:
  lbm     - ctypes binding of the C-ABI library liblbm (include/lbm.h)
  batch   - batched heterogeneous cases in one persistent launch
  inputs  - seeded synthetic input fields (no model arithmetic)
  build   - in-tree nvcc build of the CUDA library
Imports are lazy so that ``inputs`` works without a GPU or a built library.
"""
__all__ = ["lbm", "inputs", "build"]
