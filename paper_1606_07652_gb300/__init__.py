"""GB300 (sm_103a) band-limited FMM for RBF interpolation (Zhao & Stoll, arXiv 1606.07652).

The compute path is the C-ABI library ``librbf.so`` (hand-written CUDA, see
``include/rbf.h``); this package is a thin ctypes binding with the same names.
PyTorch supplies device memory and streams only.  There is no CPU fallback:
importing the binding raises when the library is missing.
"""
from ._lib import (FP32, FP64, GAUSSIAN, GRID_NESTED, GRID_SHARED, IMQ, MQ, WENDLAND, Evaluator,
                   RbfError, Tree,
                   check_device_waits, direct_sum, fmm_matvec,
                   fmm_matvec_host, interp_solve, library_path, load, profile, profile_read,
                   tree_build, version)

__all__ = ["FP32", "FP64", "GAUSSIAN", "GRID_NESTED", "GRID_SHARED", "IMQ", "MQ", "WENDLAND",
           "Evaluator", "RbfError", "Tree",
           "check_device_waits",
           "direct_sum", "fmm_matvec",
           "fmm_matvec_host", "interp_solve", "library_path", "load", "profile",
           "profile_read", "tree_build", "version"]
