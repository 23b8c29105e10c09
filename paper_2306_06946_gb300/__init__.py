"""GB300 (sm_103a) implementation of the fast constraint-matrix update for
implicit contact resolution (arXiv 2306.06946, Sec. 5, Alg. 3).

The work happens in ``libicr.so`` (CUDA C++, C ABI in include/icr.h).
``icr`` is its ctypes binding, ``driver`` strings the calls of one time step
together, ``build`` compiles the library in-tree with nvcc.
"""
from . import icr  # noqa: F401
from .icr import FP32, FP64, Context, IcrError, Scene  # noqa: F401
