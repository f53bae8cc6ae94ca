"""Restarted block GMRes with block Givens QR, plain FP64 (Ch. 5, Ch. 9.1).

Follows Alg. "bgmres" (Ch. 5.1) with M = I:
  * V^0 sigma^0 = Norm(R^0) (Householder normalizer);
  * Arnoldi step W = A V^k, orthogonalised against V^0..V^k either by block
    modified Gram-Schmidt (Alg. "block-arnoldi") or by classical block
    Gram-Schmidt repeated twice (CGS2, Ch. 9.1: all projections of one pass
    in one batch, #it = 2), then V^{k+1}, gamma = Norm(W); or the whole
    basis kept as a distributed S-QR decomposition over row tiles by the
    localized Arnoldi method (Ch. 9.3, ``localized.py``), whose global
    R-factor gives the Hessenberg column and gamma at once;
  * the new Hessenberg column is rotated by the previous block Givens factors
    Q_0 .. Q_{k-1}, then the 2s x s block [h_kk; gamma] is QR-factorised by
    Householder (full 2s x 2s Q_k), and [sigma^k; sigma^{k+1}] <- Q_k^T [sigma^k; 0];
  * stop when max_i ||sigma^{k+1} e_i|| / ||R^0_i|| <= tol (the per-column
    residual norms; ||R^k||_F = ||sigma^{k+1}||_F, Ch. 5.1);
  * back-substitution over the steps actually taken, X += sum_j V^j zeta_j,
    restart with X as the new initial guess.

Readings: the algorithm prints eta_jk = -<V^j, V^{k+1}> and V^{k+1} += V^j eta_jk,
while the Hessenberg matrix needs +<.,.>; we store h_jk = <V^j, W> and update
W -= V^j h_jk.  The back-substitution is printed up to k_max - 1 even after an
early break; we run it over the steps taken.  The Householder reflections of
the block Givens step use the same convention as ``householder_qr`` but
without the final sign fix (any QR of [h_kk; gamma] is valid; X is invariant).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from .bcg import BCGResult
from .blockops import col_norms, normalizer, spmm, stop_measure
from .localized import LocalizedArnoldi


def _full_householder_qr(M: np.ndarray):
    """Q (m x m, product of s reflectors) and R (s x s) with M = Q [R; 0]."""
    A = np.array(M, dtype=np.float64, copy=True)
    m, s = A.shape
    Q = np.eye(m)
    for j in range(s):
        x = A[j:, j]
        alpha = x[0]
        tail = float(x[1:] @ x[1:])
        if tail == 0.0:
            continue
        norm = np.sqrt(alpha * alpha + tail)
        beta = -norm if alpha >= 0 else norm
        tau = (beta - alpha) / beta
        v = x / (alpha - beta); v[0] = 1.0
        A[j:, j:] -= tau * np.outer(v, v @ A[j:, j:])
        A[j + 1:, j] = 0.0
        Q[:, j:] -= tau * np.outer(Q[:, j:] @ v, v)
    return Q, np.triu(A[:s, :])


def bgmres(A, B: np.ndarray, X0=None, tol: float = 1e-8, restart: int = 30, maxit: int = 1000,
           ortho: str = "mgs", apply_A=None, tile_rows: int = 2048, fanin: int = 2,
           norm: str = "max") -> BCGResult:
    """Alg. "bgmres" with restart length ``restart``; ``maxit`` counts Arnoldi steps.

    ortho: "mgs", "cgs2" or "localized" (row tiles of ``tile_rows`` rows, a tree of
    ``fanin`` children per node)."""
    B = np.asarray(B, dtype=np.float64)
    n, s = B.shape
    op = apply_A if apply_A is not None else (lambda V: spmm(A, V))
    X = np.zeros((n, s)) if X0 is None else np.array(X0, dtype=np.float64, copy=True)
    R = B - op(X)
    n0 = col_norms(R)
    n0_safe = np.where(n0 > 0, n0, 1.0)
    out = BCGResult(X, 0, 0, False, "ok", np.ones(s))
    total = 0
    while total < maxit:
        R = B - op(X)
        if ortho == "localized":
            la = LocalizedArnoldi(n, s, tile_rows, fanin)
            V0, sig0 = la.extend(R)
        else:
            V0, sig0 = normalizer(R)
        m = min(restart, maxit - total)
        V = [V0]
        H = np.zeros(((m + 1) * s, m * s))
        G = []                                 # block Givens factors Q_j (2s x 2s)
        sig = np.zeros(((m + 1) * s, s)); sig[:s] = sig0
        k_done = 0
        conv = False
        for k in range(m):
            W = op(V[k])
            h = np.zeros(((k + 2) * s, s))
            if ortho == "mgs":
                for j in range(k + 1):
                    hj = V[j].T @ W
                    W = W - V[j] @ hj
                    h[j * s:(j + 1) * s] = hj
            elif ortho == "cgs2":
                for _ in range(2):
                    Vk = np.hstack(V)
                    hp = Vk.T @ W
                    W = W - Vk @ hp
                    h[:(k + 1) * s] += hp
            elif ortho != "localized":
                raise ValueError(ortho)
            if ortho == "localized":
                Vn, col = la.extend(W)
                h[:] = col
            else:
                Vn, gamma = normalizer(W)
                h[(k + 1) * s:] = gamma
            for j in range(k):
                blk = h[j * s:(j + 2) * s]
                h[j * s:(j + 2) * s] = G[j].T @ blk
            Qk, rk = _full_householder_qr(h[k * s:(k + 2) * s])
            G.append(Qk)
            h[k * s:(k + 1) * s] = rk
            h[(k + 1) * s:(k + 2) * s] = 0.0
            H[:(k + 2) * s, k * s:(k + 1) * s] = h
            pair = np.vstack([sig[k * s:(k + 1) * s], np.zeros((s, s))])
            sig[k * s:(k + 2) * s] = Qk.T @ pair
            V.append(Vn)
            k_done = k + 1
            total += 1
            relres = np.where(n0 > 0, col_norms(sig[(k + 1) * s:(k + 2) * s]) / n0_safe, 0.0)
            out.history.append(stop_measure(relres, n0, norm))
            out.relres = relres
            if stop_measure(relres, n0, norm) <= tol:
                conv = True
                break
        # block back-substitution  R zeta = sigma  over the k_done steps
        zeta = [None] * k_done
        for l in range(k_done - 1, -1, -1):
            rhs = sig[l * s:(l + 1) * s].copy()
            for j in range(l + 1, k_done):
                rhs -= H[l * s:(l + 1) * s, j * s:(j + 1) * s] @ zeta[j]
            zeta[l] = np.linalg.solve(H[l * s:(l + 1) * s, l * s:(l + 1) * s], rhs)
        for j in range(k_done):
            X += V[j] @ zeta[j]
        out.iters = total
        if conv:
            out.converged = True
            return out
    out.status = "not_converged"
    return out
