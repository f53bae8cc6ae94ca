"""Tall-skinny QR by a reduction tree of local QRs, plain FP64 (Ch. 7.3).

The block is split into P row parts X_p.  Each part is factorised locally,
X_p = Q_p sigma_p (Eq. "local-qr"); the stacked R factors are factorised
again, [sigma_1; ...; sigma_P] = [sigma~_1; ...; sigma~_P] sigma, and the
sigma~_p are scattered back so that X = [Q_1 sigma~_1; ...; Q_P sigma~_P] sigma.
Applied recursively this is a tree; ``fanin`` is the number of children of
each tree node (the thesis's MPI version is binary).  Every local QR is the
Householder normalizer of ``blockops``, so diag(sigma) >= 0 at the root.

The result must agree with one Householder QR of the whole block (the QR of
a full-rank matrix with positive diagonal is unique); this is how the tree
algebra of the GPU normalizer is tested.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from .blockops import householder_qr


def tsqr(X: np.ndarray, parts: int, fanin: int = 2):
    """Return (Y, sigma) with X = Y sigma via a tree over ``parts`` row parts."""
    X = np.asarray(X, dtype=np.float64)
    n, s = X.shape
    bounds = np.linspace(0, n, parts + 1).astype(int)
    leaves = [X[bounds[i]:bounds[i + 1]] for i in range(parts)]
    if any(l.shape[0] < s for l in leaves):
        raise ValueError("every part needs at least s rows")
    Qs, Rs = zip(*[householder_qr(l) for l in leaves])
    Y_parts, sigma = _reduce(list(Rs), fanin)
    Y = np.vstack([Qs[i] @ Y_parts[i] for i in range(parts)])
    return Y, sigma


def _reduce(Rs, fanin):
    """Tree reduction of R factors; returns the scatter factors sigma~_p and the root R."""
    s = Rs[0].shape[0]
    if len(Rs) == 1:
        return [np.eye(s)], Rs[0]
    groups = [Rs[i:i + fanin] for i in range(0, len(Rs), fanin)]
    node_Q, node_R = [], []
    for g in groups:
        Qg, Rg = householder_qr(np.vstack(g))
        node_Q.append(Qg); node_R.append(Rg)
    up, root = _reduce(node_R, fanin)
    out = []
    for gi, g in enumerate(groups):
        T = node_Q[gi] @ up[gi]           # (len(g) s) x s
        for j in range(len(g)):
            out.append(T[j * s:(j + 1) * s])
    return out, root
