"""Block CG with adaptive residual re-orthonormalisation, plain FP64 (Ch. 4).

``bcg`` follows Alg. "bcgaro" (BCG-ARO, Ch. 4.3) in the grouping of
Alg. "2R-CG" (Ch. 8.1), which the thesis states is arithmetically identical.
The preconditioner M is optional (M = I when none is given, so Z = R-bar):
Z = M^{-1} R-bar, rho = <Z, R-bar>, P = Z + P beta (Alg. "bcgaro").

Readings (the thesis is silent or ambiguous here):
  * residual R = B - A X (the algorithms' sign; Ch. 4.1);
  * convergence: max over columns of ||R_i|| / ||R^0_i|| <= tol (the thesis
    uses the max-column norm, Ch. 4.1; "relative" is our reading).  Columns
    with ||R^0_i|| = 0 count as converged;
  * re-orthonormalisation criterion: see ``blockops.reortho_decision``;
  * ||R_i|| = ||R-bar sigma_i||: with re-orthonormalisation this is the column
    norm of sigma (the thesis prints Q^k, meaning R-bar^k); without it,
    sqrt((sigma^T G sigma)_ii) with the Euclidean Gram G = R-bar^T R-bar, which
    is rho when M = I and a Gram of its own otherwise (rho = R-bar^T M^{-1} R-bar);
  * beta = rho_k^{-1} gamma^T rho_{k+1} as printed in Alg. "bcgro";
  * alpha and rho are formed as upper triangles and mirrored;
  * breakdown (Cholesky of alpha or rho fails) stops with the current X.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .blockops import (Breakdown, chol_solve, cholesky_qr2, col_norms, gram, kappa_d, normalizer,
                       project_subalgebra, reortho_decision, spmm, stop_measure)
from .precond import apply_diagonal


@dataclass
class BCGResult:
    X: np.ndarray
    iters: int
    reorths: int
    converged: bool
    status: str                      # "ok", "not_converged", "breakdown"
    relres: np.ndarray               # final per-column relative residual (from sigma/rho)
    history: list = field(default_factory=list)    # max relative residual per iteration
    decisions: list = field(default_factory=list)  # re-orthonormalised in iteration k?
    kappas: list = field(default_factory=list)     # kappa_D(alpha^k) when 0 < eta < inf, else None
    alphas: list = field(default_factory=list)     # alpha^k (projected), when record_alpha
    iterates: list = field(default_factory=list)   # X^{k+1} for the first record_iterates steps
    reorths_cholqr: int = 0          # re-orthonormalisations done by CholeskyQR2 (qr="cholqr2")
    replacements: int = 0            # 1R-BCG: direct recomputations of Q and alpha


def bcg(A, B: np.ndarray, X0: np.ndarray | None = None, tol: float = 1e-8, maxit: int = 1000,
        eta: float = math.inf, p: int | None = None, forced=None, record_iterates: int = 0,
        dtype=np.float64, eps: float | None = None, apply_A=None, Minv=None,
        record_alpha: bool = False, norm: str = "max", qr: str = "householder") -> BCGResult:
    """Alg. "bcgaro" (2R grouping, Alg. "2R-CG") for A X = B.

    A: CSR (attributes n, row_ptr, col, val) or None when ``apply_A`` is given.
    p: block size of the *-subalgebra S_BP^p (None or s: block case S_B).
    forced: optional sequence of booleans replacing the adaptive criterion
        in iteration k (used to replay another implementation's decisions).
    dtype: arithmetic of the n x s blocks (float32 for the inner solve of
        iterative refinement); all s x s quantities stay float64.
    Minv: the preconditioner M^{-1}: None (M = I), a vector (a diagonal
        M^{-1}, e.g. ``precond.jacobi_inverse_diagonal(A)``) or a callable
        V -> M^{-1} V.  M must be symmetric positive definite (Ch. 4).
    norm: the stopping measure, "max" (max-column) or "fro" (Frobenius), see
        ``blockops.stop_measure``; the history records the same measure.
    qr: the normaliser of the re-orthonormalising iterations (Def. "normalizer"):
        "householder", or "cholqr2" (``blockops.cholesky_qr2``; the Householder QR for
        the blocks it declines; block case only).  Both give the unique normalizer of
        a full-rank block, so they differ by rounding only.
    """
    B = np.asarray(B)
    n, s = B.shape
    if qr not in ("householder", "cholqr2"):
        raise ValueError(f"unknown normaliser {qr!r}")
    if eps is None:
        eps = float(np.finfo(dtype).eps)
    op = apply_A if apply_A is not None else (lambda V: spmm(A, V, dtype=dtype))
    if Minv is None:
        prec = None
    elif callable(Minv):
        prec = lambda V: np.asarray(Minv(V), dtype=dtype)
    else:
        prec = lambda V: apply_diagonal(Minv, V, dtype)
    X = np.zeros((n, s), dtype=dtype) if X0 is None else np.array(X0, dtype=dtype, copy=True)
    B = B.astype(dtype, copy=False)

    R = B - op(X)
    n0 = col_norms(R)
    n0_safe = np.where(n0 > 0, n0, 1.0)
    if eta > 0:
        Rb, sigma = normalizer(R, p)
        Rb = Rb.astype(dtype)
    else:
        Rb, sigma = R, np.eye(s)
    G = gram(Rb, Rb, p)                 # Euclidean R-bar^T R-bar
    if prec is None:
        P, rho = Rb.copy(), G
    else:
        P = prec(Rb)                    # P^0 = M^{-1} R-bar^0
        rho = gram(P, Rb, p)            # rho^0 = <P^0, R-bar^0>
    res = _resid_from(sigma, G, p, reortho=False)
    relres = np.where(n0 > 0, res / n0_safe, 0.0)
    out = BCGResult(X, 0, 0, bool(stop_measure(relres, n0, norm) <= tol), "ok", relres)
    if out.converged:
        return out
    for k in range(maxit):
        Q = op(P)
        alpha = gram(P, Q, p)
        try:
            lam = chol_solve(alpha, rho)
        except Breakdown:
            out.status = "breakdown"; out.iters = k; return out
        lam = project_subalgebra(lam, p)
        if forced is not None and k < len(forced):
            reo = bool(forced[k])
        else:
            reo = reortho_decision(eta, alpha, eps)
        out.kappas.append(kappa_d(alpha) if 0.0 < eta < math.inf else None)
        if record_alpha:
            out.alphas.append(alpha.copy())
        # X^{k+1} = X^k + P^k lambda^k sigma^k (uses the old sigma)
        X += P @ (lam @ sigma).astype(dtype)
        Rt = Rb - Q @ lam.astype(dtype)
        if reo:
            fast = cholesky_qr2(Rt) if qr == "cholqr2" and (p is None or p == s) else None
            Rb, gamma = fast if fast is not None else normalizer(Rt, p)
            out.reorths_cholqr += fast is not None
            Rb = Rb.astype(dtype)
            sigma = gamma @ sigma
            out.reorths += 1
        else:
            Rb, gamma = Rt, np.eye(s)
        G = None if reo else gram(Rb, Rb, p)
        res = _resid_from(sigma, G, p, reortho=reo)
        relres = np.where(n0 > 0, res / n0_safe, 0.0)
        out.history.append(stop_measure(relres, n0, norm))
        out.decisions.append(reo)
        if k < record_iterates:
            out.iterates.append(X.copy())
        out.iters = k + 1
        out.relres = relres
        if stop_measure(relres, n0, norm) <= tol:
            out.converged = True
            return out
        if prec is None:
            Z = Rb
            rho_new = G if G is not None else gram(Rb, Rb, p)
        else:
            Z = prec(Rb)                # Z^{k+1} = M^{-1} R-bar^{k+1}
            rho_new = gram(Z, Rb, p)    # rho^{k+1} = <Z^{k+1}, R-bar^{k+1}>
        try:
            beta = chol_solve(rho, gamma.T @ rho_new)
        except Breakdown:
            out.status = "breakdown"; return out
        beta = project_subalgebra(beta, p)
        P = Z + P @ beta.astype(dtype)
        rho = rho_new
    out.status = "not_converged"
    return out


def bcg_1r(A, B: np.ndarray, X0: np.ndarray | None = None, tol: float = 1e-8, maxit: int = 1000,
           eta: float = math.inf, forced=None, record_iterates: int = 0, dtype=np.float64,
           eps: float | None = None, Minv=None, norm: str = "max", replace: int = 0) -> BCGResult:
    """BCG with one reduction per iteration, Alg. "1R-CG" (Ch. 8.1), block case S_B.

    Arithmetically equal to Alg. "bcgaro": with U = A Z, delta = <Z, U>, the
    next alpha follows from alpha^{k+1} = delta^{k+1} - beta^T alpha^k beta
    (Eq. "alpha_k+1" simplified with <Z^{k+1}, Q^k> = -beta^T alpha), and Q is
    updated as Q = U + Q beta instead of being recomputed as A P.  The norms,
    the re-orthonormalisation test and the readings are those of ``bcg``.

    replace: replacement of the recursive quantities (the residual-replacement idea
    of van der Vorst and Ye, 2000, applied to the recursion of Ch. 8.1): with replace
    = m > 0, after every m-th iteration, and after any iteration whose recursive
    alpha^{k+1} has a non-positive Cholesky pivot, Q = A P and alpha = <P, Q> are
    formed directly as in the two-reduction schedule (one more operator application);
    ``replacements`` counts them.  0: the plain recursion.
    """
    B = np.asarray(B)
    n, s = B.shape
    if eps is None:
        eps = float(np.finfo(dtype).eps)
    op = lambda V: spmm(A, V, dtype=dtype)
    if Minv is None:
        prec = lambda V: np.array(V, dtype=dtype, copy=True)
    elif callable(Minv):
        prec = lambda V: np.asarray(Minv(V), dtype=dtype)
    else:
        prec = lambda V: apply_diagonal(Minv, V, dtype)
    X = np.zeros((n, s), dtype=dtype) if X0 is None else np.array(X0, dtype=dtype, copy=True)
    B = B.astype(dtype, copy=False)

    R = B - op(X)
    n0 = col_norms(R)
    n0_safe = np.where(n0 > 0, n0, 1.0)
    if eta > 0:
        Rb, sigma = normalizer(R)
        Rb = Rb.astype(dtype)
    else:
        Rb, sigma = R, np.eye(s)
    G = gram(Rb, Rb)
    P = prec(Rb)                        # P^0 = M^{-1} R-bar^0
    rho = gram(P, Rb)                   # rho^0 = <P^0, R-bar^0>
    Q = op(P)                           # Q^0 = A P^0
    alpha = gram(P, Q)                  # alpha^0 = <P^0, Q^0>
    res = _resid_from(sigma, G, None, reortho=False)
    relres = np.where(n0 > 0, res / n0_safe, 0.0)
    out = BCGResult(X, 0, 0, bool(stop_measure(relres, n0, norm) <= tol), "ok", relres)
    if out.converged:
        return out
    for k in range(maxit):
        try:
            lam = chol_solve(alpha, rho)
        except Breakdown:
            out.status = "breakdown"; out.iters = k; return out
        if forced is not None and k < len(forced):
            reo = bool(forced[k])
        else:
            reo = reortho_decision(eta, alpha, eps)
        Rt = Rb - Q @ lam.astype(dtype)
        sigma_old = sigma
        if reo:
            Rb, gamma = normalizer(Rt)
            Rb = Rb.astype(dtype)
            sigma = gamma @ sigma
            out.reorths += 1
            G = None
        else:
            Rb, gamma = Rt, np.eye(s)
            G = gram(Rb, Rb)
        res = _resid_from(sigma, G, None, reortho=reo)
        X += P @ (lam @ sigma_old).astype(dtype)       # X^{k+1} = X^k + P^k lambda^k sigma^k
        Z = prec(Rb)                                    # Z^{k+1} = M^{-1} R-bar^{k+1}
        rho_new = gram(Z, Rb)                           # rho^{k+1} = <Z^{k+1}, R-bar^{k+1}>
        U = op(Z)                                       # U^{k+1} = A Z^{k+1}
        delta = gram(Z, U)                              # delta^{k+1} = <Z^{k+1}, U^{k+1}>
        relres = np.where(n0 > 0, res / n0_safe, 0.0)
        out.history.append(stop_measure(relres, n0, norm))
        out.decisions.append(reo)
        if k < record_iterates:
            out.iterates.append(X.copy())
        out.iters = k + 1
        out.relres = relres
        if stop_measure(relres, n0, norm) <= tol:
            out.converged = True
            return out
        try:
            beta = chol_solve(rho, gamma.T @ rho_new)
        except Breakdown:
            out.status = "breakdown"; return out
        P = Z + P @ beta.astype(dtype)
        Q = U + Q @ beta.astype(dtype)
        alpha = delta - beta.T @ alpha @ beta           # alpha^{k+1} = delta^{k+1} - beta^T alpha^k beta
        alpha = np.triu(alpha) + np.triu(alpha, 1).T
        rho = rho_new
        if replace > 0 and ((k + 1) % replace == 0 or not _chol_ok(alpha)):
            Q = op(P)                                   # Q^{k+1} = A P^{k+1}
            alpha = gram(P, Q)                          # alpha^{k+1} = <P^{k+1}, Q^{k+1}>
            out.replacements += 1
    out.status = "not_converged"
    return out


def _chol_ok(A) -> bool:
    """Whether the Cholesky factorisation of the symmetric A has positive pivots only."""
    try:
        chol_solve(A, np.eye(A.shape[0]))
        return True
    except Breakdown:
        return False


def _resid_from(sigma, G, p, reortho):
    """Column norms of the true residual R = R-bar sigma (Ch. 4.3, after Alg. "bcgro").

    G is the Euclidean Gram R-bar^T R-bar (unused after a re-orthonormalisation,
    where R-bar has orthonormal columns)."""
    if reortho:
        return col_norms(sigma)
    M = project_subalgebra(sigma.T @ G @ sigma, p)
    return np.sqrt(np.maximum(np.diag(M), 0.0))


def scalar_cg(A, b: np.ndarray, x0=None, tol: float = 1e-8, maxit: int = 1000,
              record_iterates: int = 0, apply_A=None, minv=None):
    """Textbook (preconditioned) conjugate gradients for one right-hand side (Ch. 2).

    Independent of ``bcg``: Hestenes-Stiefel with z = M^{-1} r, step length
    r.z / p.Ap and direction update z' + (r'.z' / r.z) p (M = I when ``minv``,
    the diagonal of M^{-1}, is None), stopping on ||r|| / ||r0|| <= tol.
    Returns (x, iters, history, iterates).
    """
    op = apply_A if apply_A is not None else (lambda v: spmm(A, v[:, None])[:, 0])
    pre = (lambda v: v) if minv is None else (lambda v: np.asarray(minv, dtype=np.float64) * v)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - op(x)
    z = pre(r)
    p = z.copy()
    rz = float(r @ z)
    r0 = math.sqrt(float(r @ r))
    hist, its = [], []
    if r0 == 0:
        return x, 0, hist, its
    for k in range(maxit):
        q = op(p)
        a = rz / float(p @ q)
        x = x + a * p
        r = r - a * q
        rn = math.sqrt(float(r @ r))
        hist.append(rn / r0)
        if k < record_iterates:
            its.append(x.copy())
        if rn / r0 <= tol:
            return x, k + 1, hist, its
        z = pre(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, hist, its
