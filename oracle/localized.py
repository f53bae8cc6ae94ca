"""Localized Arnoldi orthonormalisation, plain FP64 (Ch. 9.3).  Test infrastructure only.

Restates Alg. "localized-arnoldi" with its Algs. "reduction-localized" and
"back-propagation-localized".  The rows are split into tiles (the thesis's
processes).  Every tile keeps a local orthonormal basis P_p^0, P_p^1, ... of
its part of the Arnoldi basis, and the global basis vector k is
X^k_p = sum_j P_p^j (zeta_p^k)_j (Def. "Distributed S-QR decomposition").
Extending the basis by a block W:
  1. every tile orthonormalises W_p against its local basis by block modified
     Gram-Schmidt and normalises the rest (Householder): the local R-factor
     zeta~_p = [<P_p^0, W_p>; ...; <P_p^k, W_p>; r_p];
  2. a tree over the tiles (the same tree in every step; binary as printed,
     or ``fanin`` children per node) reduces the
     local R-factors: each node stacks its children's vectors, orthonormalises
     the stack against the node's own basis (modified Gram-Schmidt in the
     inner product of stacked coefficient vectors), normalises the rest and
     passes its R-factor rho = [rho_0; ...; rho_{k+1}] up; the root's rho is
     the global R-factor of W against the basis (the new Hessenberg column);
  3. back-propagation: the root hands its new basis vector's components to its
     children; a node that receives the coefficients rho~ hands
     sum_i [zeta^i_c; 0] rho~_i to child c; a tile that receives zeta_p builds
     its part of the new global basis vector X_p = sum_j P_p^j (zeta_p)_j.
The normaliser is ``blockops.normalizer`` everywhere (diag(R) >= 0), so the
global basis and R-factor are the ones of any QR with that sign convention.
"""
from __future__ import annotations

import numpy as np

from .blockops import normalizer


def _pad(v: np.ndarray, rows: int) -> np.ndarray:
    if v.shape[0] == rows:
        return v
    return np.vstack([v, np.zeros((rows - v.shape[0], v.shape[1]))])


class LocalizedArnoldi:
    """The distributed S-QR decomposition of the basis built so far (block case S_B)."""

    def __init__(self, n: int, s: int, tile_rows: int, fanin: int = 2):
        self.s = s
        self.fanin = fanin
        self.tiles = [(a, min(a + tile_rows, n)) for a in range(0, n, tile_rows)]
        if self.tiles[-1][1] - self.tiles[-1][0] < s:
            # a local S-QR needs at least s rows on every tile (local orthonormality)
            raise ValueError("the last row tile has fewer than s rows")
        self.sizes = [len(self.tiles)]
        while self.sizes[-1] > 1:
            self.sizes.append((self.sizes[-1] + fanin - 1) // fanin)
        self.P = [[] for _ in self.tiles]                    # local bases P_p^j
        self.node_basis = {(l, i): [] for l in range(1, len(self.sizes))
                           for i in range(self.sizes[l])}    # list of [zeta^i_c for c in children]

    def _children(self, l: int, i: int):
        return [c for c in range(self.fanin * i, self.fanin * (i + 1)) if c < self.sizes[l - 1]]

    def extend(self, W: np.ndarray):
        """Add the block W: returns (X^{k+1}, rho) with W = sum_j X^j rho_j over the new basis."""
        s = self.s
        k1 = len(self.P[0])                                  # basis vectors so far (k + 1)
        # 1. local modified Gram-Schmidt and normaliser on every tile
        below = []
        for p, (a, b) in enumerate(self.tiles):
            Wp = np.array(W[a:b], dtype=np.float64, copy=True)
            z = []
            for j in range(k1):
                zj = self.P[p][j].T @ Wp
                Wp = Wp - self.P[p][j] @ zj
                z.append(zj)
            Pn, r = normalizer(Wp)
            self.P[p].append(Pn)
            z.append(r)
            below.append(np.vstack(z))                       # (k1 + 1) s x s
        L = (k1 + 1) * s
        # 2. reduction up the tree (Alg. "reduction-localized")
        for l in range(1, len(self.sizes)):
            out = []
            for i in range(self.sizes[l]):
                ch = self._children(l, i)
                S = [below[c].copy() for c in ch]
                rho = []
                for comp in self.node_basis[(l, i)]:
                    zi = [_pad(v, L) for v in comp]
                    ri = sum(zi[q].T @ S[q] for q in range(len(ch)))
                    for q in range(len(ch)):
                        S[q] = S[q] - zi[q] @ ri
                    rho.append(ri)
                Q, r = normalizer(np.vstack(S))
                self.node_basis[(l, i)].append([Q[q * L:(q + 1) * L] for q in range(len(ch))])
                rho.append(r)
                out.append(np.vstack(rho))
            below = out
        rho_root = below[0]
        # 3. back-propagation (Alg. "back-propagation-localized")
        top = len(self.sizes) - 1
        if top == 0:
            coef = [np.vstack([np.zeros((k1 * s, s)), np.eye(s)])]   # one tile: its new vector
        else:
            coef = list(self.node_basis[(top, 0)][-1])               # the root's new vector
            for l in range(top - 1, 0, -1):
                nxt = []
                for i in range(self.sizes[l]):
                    rt = coef[i]
                    comps = self.node_basis[(l, i)]
                    for q in range(len(self._children(l, i))):
                        acc = np.zeros((L, s))
                        for ii, comp in enumerate(comps):
                            acc += _pad(comp[q], L) @ rt[ii * s:(ii + 1) * s]
                        nxt.append(acc)
                coef = nxt
        X = np.zeros((self.tiles[-1][1], s))
        for p, (a, b) in enumerate(self.tiles):
            zp = coef[p]
            for j in range(k1 + 1):
                X[a:b] += self.P[p][j] @ zp[j * s:(j + 1) * s]
        return X, rho_root
