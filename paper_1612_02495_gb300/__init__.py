"""GB300-native swept time-space decomposition for explicit 1D stencil solvers.

Submodules:
  swept   ctypes binding of the C-ABI library libswept.so (CUDA kernels for sm_103a)
  inputs  seeded synthetic workloads (no scheme arithmetic)

Importing the package itself loads nothing; `paper_1612_02495_gb300.swept`
raises if the CUDA library has not been built.
"""
