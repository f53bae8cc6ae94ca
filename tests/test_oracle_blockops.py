"""Pins for the oracle's block primitives (BOP, BDOT, normalizer, kappa_D, TSQR)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle.blockops import Breakdown


def test_spmm_integer_exact_against_dense():
    A = W.lap3d7(5, 4, 3)
    P = np.random.default_rng(1).integers(-50, 50, (A.n, 7)).astype(np.float64)
    Q = oracle.spmm(A, P)
    Ad = A.to_dense()
    ref = np.array([[sum(Ad[i, j] * P[j, c] for j in range(A.n)) for c in range(7)] for i in range(A.n)])
    assert np.array_equal(Q, ref)


def test_gram_brute_force_and_symmetry():
    g = np.random.default_rng(2)
    X = g.integers(-9, 9, (13, 5)).astype(float); Y = g.integers(-9, 9, (13, 5)).astype(float)
    G = oracle.gram(X, Y)
    for i in range(5):
        for j in range(5):
            a, b = min(i, j), max(i, j)
            assert G[i, j] == sum(X[r, a] * Y[r, b] for r in range(13))
    Gf = oracle.gram(X, Y, sym=False)
    for i in range(5):
        for j in range(5):
            assert Gf[i, j] == sum(X[r, i] * Y[r, j] for r in range(13))


def test_gram_subalgebra_projection():
    g = np.random.default_rng(3)
    X = g.standard_normal((20, 6))
    G = oracle.gram(X, X, p=2)
    full = X.T @ X
    for i in range(6):
        for j in range(6):
            if i // 2 == j // 2:
                assert G[i, j] == pytest.approx(full[i, j], rel=1e-14)
            else:
                assert G[i, j] == 0.0
    np.testing.assert_allclose(np.diag(oracle.gram(X, X, p=1)), np.diag(full), rtol=1e-14)


@pytest.mark.parametrize("n,s", [(40, 5), (9, 9), (300, 32), (17, 1)])
def test_householder_against_lapack(n, s):
    X = np.random.default_rng(n * s).standard_normal((n, s))
    Y, R = oracle.householder_qr(X)
    eps = np.finfo(float).eps
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.all(np.diag(R) >= 0)
    assert np.abs(Y.T @ Y - np.eye(s)).max() <= 10 * n * eps
    assert np.abs(Y @ R - X).max() <= 10 * n * eps * np.abs(X).max()
    Ql, Rl = np.linalg.qr(X)
    d = np.sign(np.diag(Rl))
    np.testing.assert_allclose(R, Rl * d[:, None], rtol=0, atol=1e-12 * np.abs(R).max())
    np.testing.assert_allclose(Y, Ql * d[None, :], rtol=0, atol=1e-11)


def test_householder_rank_deficient():
    g = np.random.default_rng(7)
    X = g.standard_normal((30, 6))
    X[:, 2] = X[:, 0] - 2 * X[:, 1]     # dependent column
    X[:, 4] = 0.0                       # zero column
    Y, R = oracle.householder_qr(X)
    assert np.abs(Y.T @ Y - np.eye(6)).max() < 1e-13
    assert np.abs(Y @ R - X).max() < 1e-13
    assert abs(R[4, 4]) < 1e-14 and abs(R[2, 2]) < 1e-13
    assert np.all(np.diag(R) >= 0)


def test_normalizer_block_parallel():
    X = np.random.default_rng(9).standard_normal((25, 6))
    Y, sig = oracle.normalizer(X, p=3)
    assert np.abs(Y @ sig - X).max() < 1e-13
    G = oracle.gram(Y, Y, p=3)
    assert np.abs(G - np.eye(6)).max() < 1e-13
    assert np.all(sig[:3, 3:] == 0) and np.all(sig[3:, :3] == 0)


def test_kappa_d_closed_forms():
    # diagonal => 1 (Ch. 4.3: "equals 1 for diagonal matrices")
    assert oracle.kappa_d(np.diag([1.0, 7.0, 1e-6])) == pytest.approx(1.0)
    # 2x2 unit-diagonal [[1,c],[c,1]]: eigenvalues 1 +- c
    for c in (0.1, -0.5, 0.99):
        M = np.array([[1.0, c], [c, 1.0]])
        assert oracle.kappa_d(M) == pytest.approx((1 + abs(c)) / (1 - abs(c)), rel=1e-12)
        D = np.diag([3.0, 0.01])     # diagonal scaling invariance
        assert oracle.kappa_d(D @ M @ D) == pytest.approx((1 + abs(c)) / (1 - abs(c)), rel=1e-12)
    assert oracle.kappa_d(np.array([[1.0, 1.0], [1.0, 1.0]])) == math.inf or \
        oracle.kappa_d(np.array([[1.0, 1.0], [1.0, 1.0]])) > 1e15


def test_reortho_decision_reading():
    eps = np.finfo(float).eps
    a_diag = np.diag([1.0, 2.0])
    assert oracle.reortho_decision(0.0, a_diag, eps) is False
    assert oracle.reortho_decision(math.inf, a_diag, eps) is True
    # kappa_D = 1: re-orthonormalise only if eta > 1/sqrt(eps)
    assert oracle.reortho_decision(1e4, a_diag, eps) is False
    assert oracle.reortho_decision(1e9, a_diag, eps) is True
    c = 1 - 1e-5    # kappa_D ~ 2e5 > 1/(1e4 sqrt(eps)) ~ 6.7e3
    assert oracle.reortho_decision(1e4, np.array([[1.0, c], [c, 1.0]]), eps) is True


def test_chol_and_lu_breakdown():
    with pytest.raises(Breakdown):
        oracle.chol_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.eye(2))
    with pytest.raises(Breakdown):
        oracle.lu_solve(np.zeros((2, 2)), np.eye(2))
    A = np.array([[4.0, 1.0], [1.0, 3.0]])
    np.testing.assert_allclose(A @ oracle.chol_solve(A, np.eye(2)), np.eye(2), atol=1e-15)


@pytest.mark.parametrize("parts,fanin", [(1, 2), (2, 2), (7, 2), (8, 3), (16, 4)])
def test_tsqr_tree_equals_single_qr(parts, fanin):
    X = np.random.default_rng(parts).standard_normal((400, 8))
    Y, sig = oracle.tsqr(X, parts, fanin)
    Y1, sig1 = oracle.householder_qr(X)
    np.testing.assert_allclose(sig, sig1, rtol=0, atol=1e-12 * np.abs(sig1).max())
    np.testing.assert_allclose(Y, Y1, rtol=0, atol=1e-12)


def test_tsqr_rank_deficient_is_valid():
    X = np.random.default_rng(4).standard_normal((200, 5))
    X[:, 3] = X[:, 1]
    Y, sig = oracle.tsqr(X, 5, 2)
    assert np.abs(Y.T @ Y - np.eye(5)).max() < 1e-13
    assert np.abs(Y @ sig - X).max() < 1e-13
    assert np.allclose(np.tril(sig, -1), 0) and np.all(np.diag(sig) >= 0)
