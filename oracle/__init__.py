"""Plain FP64 CPU oracle for the block Krylov hot path (test infrastructure).

THIS PACKAGE IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the tests
(``tests/``), ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg
of ``bench.py`` may import it.  The GPU library never calls it, and it shares
no code with the GPU library: the only common module is ``workloads`` (the
seeded problem generators, which contain none of the methods' arithmetic).

Source: N.-A. Dreier, "Hardware-Oriented Krylov Methods for High-Performance
Computing", PhD thesis, WWU Muenster 2020 (arXiv 2104.02494).  Every function
cites the chapter / algorithm / equation it restates.  The code is written for
a reader who checks it against the thesis by eye: library primitives (sparse
matrix product, dense matmul, Cholesky, LU, eigvalsh) serve as single steps,
and no blocking, fusion or reordering beyond the thesis's own is applied.

Readings of passages that are ambiguous or garbled in the thesis (residual
sign, norm, re-orthonormalisation criterion, BBiCGStab index slips, BGMRes
sign and back-substitution range) are listed in the module docstrings where
they are used.

Parity pins (checked by ``tests/test_oracle_*.py`` without a GPU): dense direct
solves, closed-form eigenvalues, LAPACK QR after sign fixing, Galerkin and
A-conjugacy invariants, block CG at s = 1 against textbook scalar CG (and preconditioned CG),
the energy minimisation over the preconditioned block Krylov space, finite
termination in ceil(n/s) steps, the Chebyshev error bound, BGMRes monotone
residuals and its column-wise least-squares characterisation, the commutation
of the block methods with a change of basis of the right-hand sides,
rank-deficient right-hand sides, finite differences for the adjoint, and
planted one-token mistakes that every battery must reject.  Functions without such a pin
are marked "parity unpinned" in their docstring (none at present).
"""
from .blockops import (spmm, gram, householder_qr, cholesky_qr2, normalizer, kappa_d, chol_solve,
                       lu_solve, col_norms, reortho_decision, project_subalgebra)
from .bcg import bcg, bcg_1r, scalar_cg, BCGResult
from .bbicgstab import bbicgstab
from .bgmres import bgmres
from .tsqr import tsqr
from .ir import bcg_ir
from .precond import jacobi_inverse_diagonal, apply_diagonal
from .localized import LocalizedArnoldi
from .adjoint import dense_adjoint, adjoint_scatter, edge_theta_grad

__all__ = [
    "spmm", "gram", "householder_qr", "cholesky_qr2", "normalizer", "kappa_d", "chol_solve", "lu_solve",
    "col_norms", "reortho_decision", "project_subalgebra", "bcg", "bcg_1r", "scalar_cg",
    "BCGResult", "bbicgstab", "bgmres", "tsqr", "bcg_ir", "dense_adjoint",
    "adjoint_scatter", "edge_theta_grad", "jacobi_inverse_diagonal", "apply_diagonal", "LocalizedArnoldi",
]
