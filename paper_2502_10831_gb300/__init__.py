"""pi/12 piecewise trigonometry of arXiv 2502.10831 on GB300 (sm_103a).

The arithmetic lives in the CUDA C-ABI library libptrig (include/ptrig.h);
this package is its thin Python layer:

  binding     ctypes binding, same names as the C entry points
  functional  tensor API (sin, cos, tan, sincos, taylor, derivative) + autograd
  workloads   seeded synthetic angle workloads
  build       nvcc build of libptrig.so

Nothing here computes a trigonometric value itself; without the built library
the calls raise ImportError.
"""
from .functional import (cos, cudamath, derivative, forward, segment, sin, sincos,  # noqa: F401
                         sincostan_loss, tan, taylor)
