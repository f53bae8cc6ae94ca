"""Block-vector building blocks of the thesis's framework, in plain FP64.

Thesis Ch. 3.2-3.3 names three kernels — BOP (apply the operator to a block),
BDOT (block inner product, an s x s element of the *-subalgebra) and BAXPY
(block update X + Y sigma) — plus the normalizer (Def. "normalizer", Ch. 3.1,
computed by Householder QR, Ch. 3.2).  This file restates each one directly.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.sparse


class Breakdown(Exception):
    """An s x s coefficient matrix could not be factorised (see Ch. 4.3)."""


def _as_scipy(A, dtype=np.float64):
    n = int(A.n)
    return scipy.sparse.csr_matrix(
        (np.asarray(A.val, dtype=dtype), np.asarray(A.col), np.asarray(A.row_ptr)), shape=(n, n))


def spmm(A, P: np.ndarray, dtype=np.float64) -> np.ndarray:
    """BOP: Q = A P for a CSR matrix A and an n x s block P (Ch. 3.3, Table "kernels").

    Each output entry is the row sum over the stored non-zeros in CSR order.
    ``dtype`` selects the arithmetic (float32 only for the inner solve of
    iterative refinement).
    """
    return np.asarray(_as_scipy(A, dtype) @ np.asarray(P, dtype=dtype))


def project_subalgebra(M: np.ndarray, p: int | None) -> np.ndarray:
    """Orthogonal projection of an s x s matrix onto S_BP^p (Def. "subalgebras", Ch. 3.1).

    S_BP^p holds the block-diagonal matrices with q = s/p diagonal blocks of
    size p x p.  p = s is the block case S_B (nothing is dropped), p = 1 the
    parallel case S_P (only the diagonal is kept).
    """
    s = M.shape[0]
    if p is None or p == s:
        return M
    assert s % p == 0
    out = np.zeros_like(M)
    for b in range(0, s, p):
        out[b:b + p, b:b + p] = M[b:b + p, b:b + p]
    return out


def gram(X: np.ndarray, Y: np.ndarray, p: int | None = None, sym: bool = True) -> np.ndarray:
    """BDOT: the block inner product <X, Y>_S = X^T Y projected to S (Ch. 3.1, Ch. 3.3).

    For the symmetric Grams of BCG (alpha = P^T A P, rho = R^T R, Eqs.
    "cg_alpha", "cg_rho") only the upper triangle is formed and mirrored,
    which both halves the work and makes the result exactly symmetric.
    Float32 inputs are multiplied and summed in float64.
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    G = X.T @ Y
    if sym:
        G = np.triu(G) + np.triu(G, 1).T
    return project_subalgebra(G, p)


def col_norms(X: np.ndarray) -> np.ndarray:
    """Euclidean norm of every column (the thesis's max-column norm, Ch. 4.1)."""
    X = np.asarray(X, dtype=np.float64)
    return np.sqrt(np.einsum("ij,ij->j", X, X))


def stop_measure(relres: np.ndarray, n0: np.ndarray, norm: str = "max") -> float:
    """Relative residual that the stopping test compares with tol (Ch. 4.1 prints
    "break if ||R|| < tol" without naming the norm; reading c2).

    relres_i = ||R_i|| / ||R^0_i|| (0 for columns with R^0_i = 0), n0_i = ||R^0_i||.
    "max": max_i relres_i, a reduction by tol in every column (the default);
    "fro": ||R||_F / ||R^0||_F = sqrt(sum_i (relres_i n0_i)^2) / sqrt(sum_i n0_i^2).
    """
    relres = np.asarray(relres, dtype=np.float64)
    if norm == "max":
        return float(relres.max(initial=0.0))
    if norm == "fro":
        n0 = np.asarray(n0, dtype=np.float64)
        den = math.sqrt(float(np.sum(n0 * n0)))
        return math.sqrt(float(np.sum((relres * n0) ** 2))) / den if den > 0 else 0.0
    raise ValueError(norm)


def householder_qr(X: np.ndarray):
    """Householder QR  X = Y sigma  with Y^T Y = I, sigma upper triangular, diag(sigma) >= 0.

    This is the normalizer of the block case (Def. "normalizer" and the
    remark after it: the thesis computes it with LAPACK xGEQRF, i.e.
    Householder reflections, because Gram-Schmidt fails for rank-deficient
    blocks).  Column j is reflected onto beta_j e_j with
    beta_j = -sign(x_1) ||x||; a column whose sub-diagonal part is already zero
    gets the identity reflector.  Y is the first s columns of H_1 ... H_s,
    so it is orthonormal even when X is rank deficient.  Finally the signs of
    the rows of sigma (and columns of Y) are flipped so that diag(sigma) >= 0,
    which makes the factorisation unique for full-rank X.
    """
    A = np.array(X, dtype=np.float64, copy=True)
    n, s = A.shape
    if n < s:
        raise ValueError("householder_qr needs n >= s")
    vs, taus = [], []
    for j in range(s):
        x = A[j:, j]
        alpha = x[0]
        tail = float(np.dot(x[1:], x[1:]))
        if tail == 0.0:
            v = np.zeros_like(x); v[0] = 1.0
            tau = 0.0
            beta = alpha
        else:
            norm = math.sqrt(alpha * alpha + tail)
            beta = -norm if alpha >= 0 else norm
            tau = (beta - alpha) / beta
            v = x / (alpha - beta)
            v[0] = 1.0
        # apply H_j = I - tau v v^T to the trailing columns
        if tau != 0.0 and j + 1 < s:
            w = v @ A[j:, j + 1:]
            A[j:, j + 1:] -= tau * np.outer(v, w)
        A[j, j] = beta
        A[j + 1:, j] = 0.0
        vs.append(v); taus.append(tau)
    R = np.triu(A[:s, :])
    # Y = H_1 ... H_s [I_s; 0], applied right to left
    Y = np.zeros((n, s)); Y[:s, :s] = np.eye(s)
    for j in range(s - 1, -1, -1):
        if taus[j] != 0.0:
            v = vs[j]
            w = v @ Y[j:, :]
            Y[j:, :] -= taus[j] * np.outer(v, w)
    d = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Y * d[None, :], R * d[:, None]


def cholesky_qr2(X: np.ndarray, min_sine2: float = 1e-10):
    """X = Y sigma by CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto,
    "CholeskyQR2: a simple and communication-avoiding algorithm for computing a
    tall-skinny QR factorization", 2014), or None when X is too close to rank
    deficient for it.

    The normalizer (Def. "normalizer") of a full-rank block is unique once
    diag(sigma) > 0, so any QR method gives it up to rounding; this one runs in
    two Gram-and-triangular passes:
        G1 = X^T X,  R1 = chol(G1) (upper, R1^T R1 = G1),  Y1 = X R1^{-1},
        G2 = Y1^T Y1, R2 = chol(G2),                       Y  = Y1 R2^{-1},
        sigma = R2 R1.
    One pass leaves Y1 with an orthogonality error of order eps kappa(X)^2; the
    second brings it to O(eps) when kappa(X) is well below eps^{-1/2}.  The
    block is declined (None) unless every pivot of the first Cholesky keeps
    R1_jj^2 > min_sine2 G1_jj: R1_jj^2 / G1_jj is the squared sine between
    column j and the span of the columns before it, so rank-deficient and
    nearly dependent blocks go to the Householder normaliser instead.  The
    second Cholesky must keep R2_jj^2 > G2_jj / 2 (G2 is then close to I).
    """
    X = np.asarray(X, dtype=np.float64)
    n, s = X.shape
    if n < s:
        raise ValueError("cholesky_qr2 needs n >= s")

    def chol_upper(G, floor):
        R = np.zeros_like(G)
        for j in range(s):
            d = G[j, j] - float(np.dot(R[:j, j], R[:j, j]))
            if not (d > floor * G[j, j]) or not (G[j, j] > 0):
                return None
            R[j, j] = math.sqrt(d)
            for c in range(j + 1, s):
                R[j, c] = (G[j, c] - float(np.dot(R[:j, j], R[:j, c]))) / R[j, j]
        return R

    G1 = X.T @ X
    R1 = chol_upper(G1, min_sine2)
    if R1 is None:
        return None
    Y1 = np.linalg.solve(R1.T, X.T).T          # X R1^{-1}
    G2 = Y1.T @ Y1
    R2 = chol_upper(G2, 0.5)
    if R2 is None:
        return None
    Y = np.linalg.solve(R2.T, Y1.T).T
    return Y, R2 @ R1


def normalizer(X: np.ndarray, p: int | None = None):
    """Y, sigma = Norm_S(X) (Def. "normalizer"): Householder QR of every p-column group.

    For S_B (p = s) this is one QR of the whole block; for S_BP^p it is q
    independent QRs, and sigma is block diagonal.
    """
    X = np.asarray(X, dtype=np.float64)
    n, s = X.shape
    if p is None or p == s:
        return householder_qr(X)
    Y = np.zeros_like(X); sig = np.zeros((s, s))
    for b in range(0, s, p):
        Yb, Rb = householder_qr(X[:, b:b + p])
        Y[:, b:b + p] = Yb; sig[b:b + p, b:b + p] = Rb
    return Y, sig


def kappa_d(alpha: np.ndarray) -> float:
    """Diagonally scaled condition number kappa(delta^-1/2 alpha delta^-1/2) (Def. in Ch. 4.3).

    delta = diag(alpha).  The condition number is the 2-norm one, i.e. the
    ratio of the extreme eigenvalues of the scaled symmetric matrix.  A
    non-positive diagonal entry or eigenvalue gives +inf.
    """
    d = np.diag(alpha).astype(np.float64)
    if np.any(d <= 0):
        return math.inf
    r = 1.0 / np.sqrt(d)
    M = alpha * r[:, None] * r[None, :]
    ev = np.linalg.eigvalsh(M)
    if ev[0] <= 0:
        return math.inf
    return float(ev[-1] / ev[0])


def reortho_decision(eta: float, alpha: np.ndarray, eps: float) -> bool:
    """Adaptive re-orthonormalisation criterion (Eq. "reortho_criterion", Ch. 4.3).

    As printed, eta * kappa_D > sqrt(eps) holds for every eta >= sqrt(eps)
    (kappa_D >= 1), which contradicts the thesis's own Table
    "it_count_reortho" (eta = 0.1 re-orthonormalises 3 times in 146
    iterations).  Reading used here: re-orthonormalise when
    eta * kappa_D(alpha) > 1 / sqrt(eps), so eta = 0 never, eta = inf always,
    and a larger eta more often.  eps is the machine epsilon of the working
    precision.
    """
    if eta == 0:
        return False
    if math.isinf(eta):
        return True
    return eta * kappa_d(alpha) > 1.0 / math.sqrt(eps)


def chol_solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A^{-1} B for a symmetric positive definite s x s A, via Cholesky (used for lambda, beta)."""
    try:
        L = np.linalg.cholesky(A)
    except np.linalg.LinAlgError as e:
        raise Breakdown("Cholesky factorisation failed") from e
    Y = scipy.linalg.solve_triangular(L, B, lower=True)
    return scipy.linalg.solve_triangular(L.T, Y, lower=False)


def lu_solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A^{-1} B for a general s x s A (LU with partial pivoting), used by BBiCGStab."""
    try:
        X = np.linalg.solve(A, B)
    except np.linalg.LinAlgError as e:
        raise Breakdown("singular coefficient matrix") from e
    if not np.all(np.isfinite(X)):
        raise Breakdown("non-finite coefficient matrix")
    return X
