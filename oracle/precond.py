"""Preconditioners M^{-1} for the oracle's BCG (Ch. 2, Ch. 4).  Test infrastructure only.

Ch. 2 names the splitting preconditioners, of which the Jacobi method takes
the diagonal of A; Ch. 4 requires M symmetric positive definite.  Point Jacobi
is M = diag(A), kept here as the vector diag(A)^{-1}: M^{-1} V scales row i of
V by its i-th entry.
"""
from __future__ import annotations

import numpy as np


def jacobi_inverse_diagonal(A) -> np.ndarray:
    """diag(A)^{-1} of a CSR matrix (the stored entries with column == row, summed)."""
    n = int(A.n)
    rp = np.asarray(A.row_ptr, dtype=np.int64)
    col = np.asarray(A.col, dtype=np.int64)
    val = np.asarray(A.val, dtype=np.float64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    on = col == rows
    d = np.zeros(n)
    np.add.at(d, rows[on], val[on])
    if not np.all(np.isfinite(d)) or np.any(d == 0.0):
        raise ValueError("A has a zero or non-finite diagonal entry")
    return 1.0 / d


def apply_diagonal(minv: np.ndarray, V: np.ndarray, dtype=np.float64) -> np.ndarray:
    """M^{-1} V for a diagonal M^{-1} given by its entries, in ``dtype`` arithmetic."""
    w = np.asarray(minv).astype(dtype)
    return (w[:, None] * np.asarray(V, dtype=dtype)).astype(dtype, copy=False)
