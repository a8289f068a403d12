"""B300 (sm_103a) implementation of the TRED hot path (arXiv 2602.12052).

The compute lives in libtred.so (hand-written CUDA behind the C ABI of
include/tred.h); ``abi`` is its ctypes binding, ``tred`` the torch-facing wrapper
and step driver, ``build`` the nvcc build of the library.
"""
__all__ = ["abi", "build", "tred"]
