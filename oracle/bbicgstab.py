"""Block BiCGStab with adaptive residual re-orthonormalisation, plain FP64 (Ch. 6).

Follows Alg. "BlockBiCGStab_with_reortho" (Ch. 6.2) with M = I, so
Z-hat = Q-hat, V-hat = R-hat, and T-hat = V-hat - Z-hat lambda-hat equals
S-hat in the branch without re-orthonormalisation (and M^{-1} S-hat = S-hat in
the other branch): T-hat = S-hat always.

Readings of the printed algorithm:
  * the half step X^{k+1/2} uses lambda-hat^k (the printed un-hatted
    lambda^k is a slip: X^{k+1/2} = X^k + P-hat lambda-hat sigma^k follows
    from sigma^k lambda^k = lambda-hat^k sigma^k);
  * the full step uses sigma^{k+1} (= sigma^k when no re-orthonormalisation
    happens), because T-hat is expressed in the new transformation
    (S = S-hat sigma^{k+1});
  * the derivation's "+ omega Z" is the algorithm's "- omega Z";
  * the break test uses the true residual R-hat^{k+1} sigma^{k+1}, whose
    column norms come from the Gram R-hat^T R-hat; that Gram is also the
    one kappa_D is evaluated on in the next iteration;
  * omega-hat minimises the transformed residual, as the thesis defines it;
  * shadow block M^{-T} R~0 = P-hat^0 (the thesis's suggested choice);
  * criterion: eta * kappa_D(R-hat^T R-hat) > 1/sqrt(eps) (see
    ``blockops.reortho_decision``); eta != 0 also normalises R^0;
  * a singular shadow Gram R~0^T Q-hat or <U,U>_F = 0 is a breakdown.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from .bcg import BCGResult
from .blockops import (Breakdown, col_norms, gram, lu_solve, normalizer, reortho_decision, spmm,
                       stop_measure)


def bbicgstab(A, B: np.ndarray, X0=None, tol: float = 1e-8, maxit: int = 1000,
              eta: float = 100.0, forced=None, record_iterates: int = 0, apply_A=None,
              eps: float | None = None, norm: str = "max") -> BCGResult:
    B = np.asarray(B, dtype=np.float64)
    n, s = B.shape
    eps = float(np.finfo(np.float64).eps) if eps is None else eps
    op = apply_A if apply_A is not None else (lambda V: spmm(A, V))
    X = np.zeros((n, s)) if X0 is None else np.array(X0, dtype=np.float64, copy=True)

    R = B - op(X)
    n0 = col_norms(R)
    n0_safe = np.where(n0 > 0, n0, 1.0)
    if eta != 0:
        Rh, sigma = normalizer(R)
    else:
        Rh, sigma = R, np.eye(s)
    Ph = Rh.copy()
    R0s = Ph.copy()            # shadow block, fixed for the whole solve
    rhoRR = gram(Rh, Rh)
    out = BCGResult(X, 0, 0, False, "ok", np.ones(s))
    for k in range(maxit):
        Qh = op(Ph)
        Gq = gram(R0s, Qh, sym=False)
        try:
            lam = lu_solve(Gq, gram(R0s, Rh, sym=False))
        except Breakdown:
            out.status = "breakdown"; out.iters = k; return out
        Sh = Rh - Qh @ lam
        X += Ph @ (lam @ sigma)
        if forced is not None and k < len(forced):
            reo = bool(forced[k])
        else:
            reo = reortho_decision(eta, rhoRR, eps)
        if reo:
            Sh, gamma = normalizer(Sh)
            sigma_new = gamma @ sigma
            out.reorths += 1
        else:
            sigma_new = sigma
        Th = Sh
        Uh = op(Th)
        uu = float(np.sum(Uh * Uh))
        if uu == 0.0 or not math.isfinite(uu):
            out.status = "breakdown"; out.iters = k + 1; return out
        omega = float(np.sum(Uh * Sh)) / uu
        X += omega * (Th @ sigma_new)
        Rh = Sh - omega * Uh
        rhoRR = gram(Rh, Rh)
        M = sigma_new.T @ rhoRR @ sigma_new
        relres = np.where(n0 > 0, np.sqrt(np.maximum(np.diag(M), 0.0)) / n0_safe, 0.0)
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
            beta = -lu_solve(Gq, gram(R0s, Uh, sym=False))
        except Breakdown:
            out.status = "breakdown"; return out
        Ph = Rh + (Ph - omega * Qh) @ beta
        sigma = sigma_new
    out.status = "not_converged"
    return out
