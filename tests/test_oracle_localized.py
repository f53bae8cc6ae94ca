"""Pins for the oracle's localized Arnoldi (Ch. 9.3) and BGMRes with it.

  * a distributed S-QR decomposition is an S-QR decomposition (the Lemma after
    Def. "Distributed S-QR decomposition"): extending by random blocks W^0, W^1,
    ... yields the Q and R of LAPACK's QR of [W^0 W^1 ...] (signs fixed to
    diag(R) >= 0), and every tile's local basis is orthonormal;
  * tiles whose rows are locally rank deficient (the Remark: the global block
    can have full rank while a tile's part does not) change nothing;
  * BGMRes with the localized method equals BGMRes with block MGS and CGS2,
    for one tile, even and odd tile counts (an unbalanced tree);
  * tiles with fewer than s rows are rejected.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle.localized import LocalizedArnoldi


def _qr_fixed(M):
    Q, R = np.linalg.qr(M)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d, R * d[:, None]


@pytest.mark.parametrize("fanin", [2, 3, 4])
@pytest.mark.parametrize("n,s,tile", [(300, 3, 300), (300, 3, 64), (301, 4, 40), (258, 2, 16)])
def test_distributed_qr_is_a_qr_of_the_concatenated_blocks(n, s, tile, fanin):
    g = np.random.default_rng(n + s + tile)
    blocks = [g.standard_normal((n, s)) for _ in range(6)]
    la = LocalizedArnoldi(n, s, tile, fanin)
    Xs, cols = [], []
    for Wb in blocks:
        X, rho = la.extend(Wb)
        Xs.append(X)
        cols.append(rho)
    Q, R = _qr_fixed(np.hstack(blocks))
    for k in range(6):
        assert np.abs(Xs[k] - Q[:, k * s:(k + 1) * s]).max() <= 1e-12
        Rk = np.zeros(((k + 1) * s, s))
        Rk[:] = R[:(k + 1) * s, k * s:(k + 1) * s]
        assert np.abs(cols[k] - Rk).max() <= 1e-12 * np.abs(R).max()
    for p, (a, b) in enumerate(la.tiles):
        # local orthonormality (Eq. "local-ortho") needs as many tile rows as basis columns;
        # a smaller tile exhausts its local space, whose further local vectors carry
        # rounding only (weighted by R-factor entries of that size, as the check above shows)
        if b - a >= 6 * s:
            Pp = np.hstack(la.P[p])
            assert np.abs(Pp.T @ Pp - np.eye(Pp.shape[1])).max() <= 1e-12


def test_locally_rank_deficient_tiles():
    n, s, tile = 240, 3, 40
    g = np.random.default_rng(4)
    blocks = [g.standard_normal((n, s)) for _ in range(4)]
    blocks[1][40:80] = 0.0                       # tile 1 sees nothing of W^1
    blocks[2][120:160, 2] = blocks[2][120:160, 0]  # tile 3: rank 2 locally
    la = LocalizedArnoldi(n, s, tile)
    Xs = [la.extend(Wb)[0] for Wb in blocks]
    Q, _ = _qr_fixed(np.hstack(blocks))
    assert np.abs(np.hstack(Xs) - Q).max() <= 1e-11


@pytest.mark.parametrize("tile,fanin", [(1000, 2), (500, 2), (200, 2), (143, 2), (64, 2), (64, 4), (64, 8)])
def test_bgmres_localized_equals_mgs_and_cgs2(tile, fanin):
    prob = W.problem("convdiff3d", grid=10)
    a = oracle.bgmres(prob.A, prob.B, tol=1e-9, restart=8, maxit=60, ortho="mgs")
    b = oracle.bgmres(prob.A, prob.B, tol=1e-9, restart=8, maxit=60, ortho="localized", tile_rows=tile,
                      fanin=fanin)
    c = oracle.bgmres(prob.A, prob.B, tol=1e-9, restart=8, maxit=60, ortho="cgs2")
    assert a.converged and b.converged and a.iters == b.iters == c.iters
    assert np.abs(b.X - a.X).max() <= 1e-10 * np.abs(a.X).max()
    assert np.abs(b.history[-1] - a.history[-1]) <= 1e-4 * a.history[-1]
    Xs = np.linalg.solve(prob.A.to_dense(), prob.B)
    true = oracle.col_norms(prob.B - oracle.spmm(prob.A, b.X)) / oracle.col_norms(prob.B)
    assert true.max() <= 1.01e-9 and np.abs(b.X - Xs).max() <= 1e-6 * np.abs(Xs).max()


def test_short_last_tile_rejected():
    with pytest.raises(ValueError):
        LocalizedArnoldi(103, 4, 50)             # last tile: 3 rows < s
