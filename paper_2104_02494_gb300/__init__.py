"""bkrylov: block Krylov solvers for one GB300 GPU (sm_103a).

Block CG with adaptive residual re-orthonormalisation, block BiCGStab,
restarted block GMRes with a TSQR normalizer, FP32 + FP64 iterative
refinement and an adjoint for reverse-mode differentiation, after
N.-A. Dreier, "Hardware-Oriented Krylov Methods for High-Performance
Computing" (2020).  All computation runs in the hand-written CUDA kernels of
``csrc/`` behind the C ABI of ``include/bkrylov.h``; this package only
marshals arguments.  Importing it does not load the library; the first
``Handle`` does, and raises if the library has not been built.
"""
from . import _lib
from .build import build

__all__ = ["build", "_lib", "Handle", "Operator", "SolveInfo", "BkError", "operator_from_problem",
           "BKrylovSolve"]


def __getattr__(name):
    if name in ("Handle", "Operator", "SolveInfo", "BkError", "operator_from_problem"):
        from . import api
        return getattr(api, name)
    if name == "BKrylovSolve":
        from . import autograd
        return autograd.BKrylovSolve
    raise AttributeError(name)
