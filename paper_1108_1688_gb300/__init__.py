"""GB300 (sm_103a) solver for the single-factor HJM model with stochastic
volatility: the Douglas ADI march of the pricing PDE as hand-written CUDA
kernels behind a C ABI (include/hjm.h).

Modules:
  hjm        ctypes binding of libhjm (same names as the C ABI)
  workloads  seeded synthetic inputs shaped like the paper's workloads
  _build     in-tree nvcc build of libhjm.so for sm_103a
"""
