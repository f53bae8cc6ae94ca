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


@pytest.mark.parametrize("s", [1, 4, 8])
def test_bcg_with_cholqr2_normaliser_matches_householder(s):
    """The normalizer of a full-rank block is unique (Def. "normalizer"), so BCG with the
    CholeskyQR2 normaliser follows the Householder one iterate for iterate up to
    rounding, re-orthonormalising in every iteration (eta = inf)."""
    import workloads as W
    prob = W.problem("poisson2d", s=s, grid=20)
    r1 = oracle.bcg(prob.A, prob.B, tol=1e-10, maxit=400, record_iterates=30)
    r2 = oracle.bcg(prob.A, prob.B, tol=1e-10, maxit=400, record_iterates=30, qr="cholqr2")
    assert r1.status == r2.status == "ok" and abs(r1.iters - r2.iters) <= 1
    for a, b in zip(r1.iterates, r2.iterates):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    assert r1.decisions == r2.decisions[:len(r1.decisions)]


def test_bcg_cholqr2_declines_nearly_dependent_residual_blocks():
    """Columns 1 and 3 of B differ by 1e-7 relative and the first two iterations keep R
    as it is (eta = 0 with forced decisions): R-tilde of iteration 2 is then nearly
    dependent (squared sine ~1e-14), CholeskyQR2 declines it and the Householder QR
    normalises; every later block is taken by CholeskyQR2.  A block that the normaliser
    made orthonormal stays far from dependent (its near-dependence moved into sigma)."""
    import workloads as W
    prob = W.problem("poisson2d", s=4, grid=16)
    B = prob.B.copy()
    B[:, 3] = B[:, 1] + 1e-7 * np.linalg.norm(B[:, 1]) * prob.B[:, 3] / np.linalg.norm(prob.B[:, 3])
    forced = [False, False] + [True] * 400
    r1 = oracle.bcg(prob.A, B, tol=1e-9, maxit=400, eta=0.0, forced=forced)
    r2 = oracle.bcg(prob.A, B, tol=1e-9, maxit=400, eta=0.0, forced=forced, qr="cholqr2")
    assert r1.status == r2.status == "ok"
    assert r2.reorths == r1.reorths and r2.reorths_cholqr == r2.reorths - 1
    X = np.linalg.solve(prob.A.toarray() if hasattr(prob.A, "toarray") else _dense(prob.A), B)
    for r in (r1, r2):
        assert np.abs(r.X - X).max() <= 1e-6 * np.abs(X).max()
    # the well-separated default case: CholeskyQR2 takes every block
    r3 = oracle.bcg(prob.A, prob.B, tol=1e-9, maxit=400, qr="cholqr2")
    assert r3.reorths_cholqr == r3.reorths == r3.iters
    assert oracle.cholesky_qr2(B) is None
    with pytest.raises(ValueError):
        oracle.bcg(prob.A, B, qr="gram-schmidt")


def _dense(A):
    D = np.zeros((A.n, A.n))
    for i in range(A.n):
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            D[i, A.col[e]] = A.val[e]
    return D
