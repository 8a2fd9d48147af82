"""GB300-native FP64 time-iterated stencils (Jacobi and Gauss-Seidel).

The compute path lives in the CUDA shared library built from ``csrc/``;
:mod:`paper_2010_04868_gb300.stencil` is the Python binding of its C ABI.
Importing this package loads nothing: the binding loads the library on first
use and raises if it is missing.
"""
__all__ = ["inputs", "stencil"]
