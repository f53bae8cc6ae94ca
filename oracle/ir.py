"""Mixed-precision iterative refinement around block CG (not in the thesis).

The thesis shows single precision needs many more iterations and
re-orthonormalisations than double (Table "it_count_reortho", Ch. 4.4); this
restates the classical refinement loop that keeps the accurate part in FP64:

    X = X0
    repeat
        R = B - A X                          (FP64)
        stop if max_i ||R_i|| / ||B_i|| <= tol
        D = inner FP32 block CG on A D = R    (relative tol ``inner_tol`` per column)
        X += D                               (FP64)

The inner right-hand side is scaled column by column by 1/||R_i|| before it
is rounded to FP32 (and D is scaled back), so its entries stay O(1) whatever
the outer residual's size; block CG with S_B is invariant under this right
scaling.  The inner solve is ``bcg`` with float32 blocks (float64 s x s
arithmetic, Grams summed in float64).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .bcg import bcg
from .blockops import col_norms, spmm, stop_measure


@dataclass
class IRResult:
    X: np.ndarray
    outer: int
    inner_iters: list = field(default_factory=list)
    relres: np.ndarray = None
    converged: bool = False


def bcg_ir(A, B: np.ndarray, tol: float = 1e-10, inner_tol: float = 1e-5, max_outer: int = 20,
           inner_maxit: int = 5000, eta: float = math.inf, Minv=None, X0=None,
           norm: str = "max") -> IRResult:
    """Refinement loop above from X0 (zero when not given); ``Minv`` (optional, see
    ``bcg``) preconditions the inner solve.  ``norm`` is the measure of the outer test
    (``blockops.stop_measure``, relative to ||B||); the inner solves keep the
    per-column test of reading c19."""
    B = np.asarray(B, dtype=np.float64)
    n, s = B.shape
    X = np.zeros((n, s)) if X0 is None else np.array(X0, dtype=np.float64, copy=True)
    nb = col_norms(B)
    nb_safe = np.where(nb > 0, nb, 1.0)
    out = IRResult(X, 0)
    for it in range(max_outer + 1):
        R = B - spmm(A, X)
        nr = col_norms(R)
        out.relres = np.where(nb > 0, nr / nb_safe, 0.0)
        if stop_measure(out.relres, nb, norm) <= tol:
            out.converged = True
            return out
        if it == max_outer:
            break
        scale = np.where(nr > 0, nr, 1.0)
        Rs = (R / scale[None, :]).astype(np.float32)
        inner = bcg(A, Rs, tol=inner_tol, maxit=inner_maxit, eta=eta, dtype=np.float32,
                    Minv=Minv)
        out.inner_iters.append(inner.iters)
        X += inner.X.astype(np.float64) * scale[None, :]
        out.outer = it + 1
    return out
