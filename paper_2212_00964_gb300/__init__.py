"""GB300-native HEX8 weak-form kernels of the differentiable FEM of JAX-FEM
(arXiv 2212.00964): residual, matrix-free tangent, adjoint VJP, Newton-PCG
solves and a batched launcher, behind the C-ABI of include/fem.h.

Modules:
  fem       -- ctypes binding of libfemgb.so (same names as the C entry points)
  autograd  -- torch.autograd.Function around fem_solve / fem_adjoint
  inputs    -- seeded synthetic workloads (no method arithmetic)
  build     -- nvcc build of libfemgb.so for sm_103a
"""
