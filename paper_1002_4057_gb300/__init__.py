"""GB300-native tiled inversion of symmetric positive definite matrices.

The compute lives in libspdinv.so (CUDA kernels for sm_103a behind the C-ABI
of include/spdinv.h).  This package is its Python binding:

  _lib     the C-ABI functions under their C names (ctypes, marshalling only)
  torch_api  thin wrappers taking torch tensors (column-major CUDA tensors),
             and the autograd Function of the inversion
  build    compiles the library in-tree

Importing the package loads nothing; the library is loaded on first use.
"""
from . import _lib  # noqa: F401
