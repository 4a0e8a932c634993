"""GB300 (sm_103a) library for the Davidson diagonalisation of DMRG superblock Hamiltonians.

The compute path is the CUDA shared library built from ``csrc/`` (C ABI in
``include/dmrg.h``); ``capi`` is its ctypes binding.  Importing this package does not
build or load anything; ``capi.load()`` raises if the library has not been built.
"""
from .capi import (DavidsonState, DmrgError, NotConverged, Plan, gemv_trans, load,  # noqa: F401
                   solve_batched)

__all__ = ["Plan", "DavidsonState", "DmrgError", "NotConverged", "gemv_trans", "load",
           "solve_batched"]
