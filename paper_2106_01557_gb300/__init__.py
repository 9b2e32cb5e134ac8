"""GB300-native (sm_103a) implementation of the fused f+g time step of the
thermal liquid-vapor lattice Boltzmann model of Huang, Wu & Adams (PRL 2021).

Submodules:
  lbm       - ctypes binding of the C-ABI library liblbm (include/lbm.h):
              single cases (Lattice), batched heterogeneous cases in one
              persistent launch (Batch), the allocation-free record
  surrogate - training data, training loop and rollout study of the
              learned surrogate (calls liblbm's lbm_surrogate_* entry points)
  inputs    - seeded synthetic input fields (no model arithmetic)
  build     - in-tree nvcc build of the CUDA library
Imports are lazy so that ``inputs`` works without a GPU or a built library.
"""
__all__ = ["lbm", "surrogate", "inputs", "build"]
