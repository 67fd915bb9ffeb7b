"""Fused BLAS-1/2 sequences (Table I of the Build to Order BLAS paper) for GB300.

Every operation runs in hand-written CUDA kernels for sm_103a inside
libbto.so; this package is the ctypes binding of its C ABI (include/bto.h),
with the C names.  PyTorch only supplies device memory and streams.
"""
from ._lib import *  # noqa: F401,F403
from ._lib import BtoError, lib, exported_symbols, OPS  # noqa: F401
