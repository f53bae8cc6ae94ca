"""Pins of the oracle's CholeskyQR2 normaliser (the GPU's fast path for well-conditioned
blocks; Def. "normalizer": the QR with diag(sigma) > 0 is unique for a full-rank block).

Pinned against the Householder normaliser (itself pinned to LAPACK), against its own
defining properties (Y^T Y = I, X = Y sigma, sigma upper triangular with a positive
diagonal) and against its decline test: rank-deficient and nearly dependent blocks are
left to the Householder path.
"""
import numpy as np
import pytest

import oracle

EPS = np.finfo(np.float64).eps


@pytest.mark.parametrize("n,s,cond", [(50, 3, 1e1), (1000, 8, 1e3), (4000, 16, 1e5), (3000, 32, 1e2),
                                      (64, 1, 1.0)])
def test_cholqr2_equals_householder(n, s, cond):
    g = np.random.default_rng(n + s)
    U, _ = np.linalg.qr(g.standard_normal((n, s)))
    V, _ = np.linalg.qr(g.standard_normal((s, s)))
    sv = np.geomspace(1.0, 1.0 / cond, s)
    X = (U * sv) @ V.T * 3.7
    out = oracle.cholesky_qr2(X)
    assert out is not None
    Y, R = out
    Yh, Rh = oracle.householder_qr(X)
    assert np.abs(Y.T @ Y - np.eye(s)).max() <= 20 * s * EPS
    assert np.abs(Y @ R - X).max() <= 20 * s * EPS * np.abs(X).max()
    assert np.array_equal(R, np.triu(R)) and (np.diag(R) > 0).all()
    # the unique positive-diagonal QR: both methods agree to ~ eps kappa
    assert np.abs(R - Rh).max() <= 50 * s * EPS * cond * np.abs(Rh).max()
    assert np.abs(Y - Yh).max() <= 50 * s * EPS * cond


def test_cholqr2_declines_deficient_blocks():
    g = np.random.default_rng(7)
    X = g.standard_normal((200, 5))
    X[:, 3] = X[:, 0] - 2 * X[:, 1]                # exactly dependent
    assert oracle.cholesky_qr2(X) is None
    X2 = g.standard_normal((200, 5))
    X2[:, 4] = X2[:, 2] + 1e-7 * g.standard_normal(200)   # sine ~ 1e-7 < 1e-5
    assert oracle.cholesky_qr2(X2) is None
    X3 = g.standard_normal((200, 5))
    X3[:, 1] = 0.0                                 # a zero column
    assert oracle.cholesky_qr2(X3) is None
    X4 = g.standard_normal((200, 5))
    X4[:, 4] = X4[:, 2] + 1e-3 * g.standard_normal(200)   # sine ~ 1e-3: accepted
    out = oracle.cholesky_qr2(X4)
    assert out is not None
    Y, R = out
    assert np.abs(Y.T @ Y - np.eye(5)).max() <= 100 * EPS


def test_cholqr2_one_pass_is_not_enough():
    # the second pass is what brings the orthogonality to eps: one pass leaves
    # ~ eps kappa^2 (pins that the oracle really runs two)
    g = np.random.default_rng(3)
    U, _ = np.linalg.qr(g.standard_normal((2000, 6)))
    V, _ = np.linalg.qr(g.standard_normal((6, 6)))
    X = (U * np.geomspace(1, 1e-5, 6)) @ V.T     # kappa 1e5, columns far from orthogonal
    G1 = X.T @ X
    R1 = np.linalg.cholesky(G1).T
    Y1 = np.linalg.solve(R1.T, X.T).T
    assert np.abs(Y1.T @ Y1 - np.eye(6)).max() > 1e-8
    Y, R = oracle.cholesky_qr2(X)
    assert np.abs(Y.T @ Y - np.eye(6)).max() <= 100 * EPS
