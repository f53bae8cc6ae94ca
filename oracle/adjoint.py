"""Adjoint (reverse-mode) derivatives of the block solve X = A^{-1} B (not in the thesis).

For a loss L(X) with G = dL/dX:
    A^T Lambda = G,     dL/dB = Lambda,     dL/dA_ij = -sum_k Lambda_ik X_jk,
the last one needed only on the sparsity pattern of A.  For the per-edge
diffusion operator A = sum_e a_e (e_i - e_j)(e_i - e_j)^T (+ a_e e_i e_i^T on
boundary edges) with a_e = exp(theta_e), the chain rule gives
    dL/dtheta_e = -a_e sum_k (Lambda_ik - Lambda_jk)(X_ik - X_jk)   (interior),
    dL/dtheta_e = -a_e sum_k Lambda_ik X_ik                          (boundary).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def dense_adjoint(Adense: np.ndarray, B: np.ndarray, Xt: np.ndarray):
    """Loss L = 0.5 ||X - Xt||^2 of X = A^{-1} B by dense solves; returns (L, X, Lambda, dA)."""
    X = np.linalg.solve(Adense, B)
    G = X - Xt
    Lam = np.linalg.solve(Adense.T, G)
    dA = -Lam @ X.T
    return 0.5 * float(np.sum(G * G)), X, Lam, dA


def adjoint_scatter(A, Lam: np.ndarray, X: np.ndarray) -> np.ndarray:
    """dL/da for every stored entry (i, j) of the CSR matrix A: -sum_k Lam_ik X_jk."""
    rows = np.repeat(np.arange(A.n), np.diff(np.asarray(A.row_ptr)))
    cols = np.asarray(A.col)
    return -np.einsum("ek,ek->e", Lam[rows], X[cols])


def edge_theta_grad(nx: int, ny: int, ax: np.ndarray, ay: np.ndarray, Lam: np.ndarray,
                    X: np.ndarray):
    """dL/dtheta for the horizontal (ny, nx+1) and vertical (ny+1, nx) edge arrays."""
    s = X.shape[1]
    L3 = Lam.reshape(ny, nx, s); X3 = X.reshape(ny, nx, s)
    gx = np.zeros_like(ax); gy = np.zeros_like(ay)
    # horizontal edges: x in 1..nx-1 interior, x = 0 and x = nx boundary
    dl = L3[:, 1:, :] - L3[:, :-1, :]; dx = X3[:, 1:, :] - X3[:, :-1, :]
    gx[:, 1:nx] = -ax[:, 1:nx] * np.sum(dl * dx, axis=2)
    gx[:, 0] = -ax[:, 0] * np.sum(L3[:, 0, :] * X3[:, 0, :], axis=1)
    gx[:, nx] = -ax[:, nx] * np.sum(L3[:, nx - 1, :] * X3[:, nx - 1, :], axis=1)
    dl = L3[1:, :, :] - L3[:-1, :, :]; dx = X3[1:, :, :] - X3[:-1, :, :]
    gy[1:ny, :] = -ay[1:ny, :] * np.sum(dl * dx, axis=2)
    gy[0, :] = -ay[0, :] * np.sum(L3[0, :, :] * X3[0, :, :], axis=1)
    gy[ny, :] = -ay[ny, :] * np.sum(L3[ny - 1, :, :] * X3[ny - 1, :, :], axis=1)
    return gx, gy
