"""Degenerate right-hand sides: rank-deficient B (a zero column, duplicated and
linearly dependent columns).

The residual re-orthonormalisation of Ch. 4.3 exists for exactly this case: the
residual block is kept as R = R-bar sigma with R-bar orthonormal, so a
rank-deficient R makes sigma singular while the iteration itself keeps a full-rank
block (the normaliser completes R-bar with further orthonormal columns) and does
not break down, where the unstabilised iteration (eta = 0) has a singular alpha.
What the mathematics fixes, and is pinned here:
  * eta = 0 with a zero column breaks down in the first iteration (alpha = P^T A P
    has an exactly zero row; so does BBiCGStab's shadow Gram);
  * with the normaliser every method converges; a zero column of B gives an
    exactly zero column of X_k for every k (its column of sigma is zero, and
    X is only ever updated through sigma); columns that are copies or linear
    combinations of others give the same copies / combinations of X_k (the
    iterate of every column is the minimiser over one common search space, a
    linear function of that column of B);
  * the search space of the stabilised run contains the block Krylov space of
    the independent columns alone, so in every step each of those columns has
    an A-energy error (BCG) resp. a residual norm (BGMRes) no larger than in a
    run on the independent columns alone (Eq. "energy-minimizer"; Ch. 5.1).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

IND = [0, 1, 3, 6]          # independent columns of the block below


def degenerate_block(B):
    """Columns 2 = 0, 4 = column 1, 5 = 0.5 col 0 - 2 col 3, 7 = -3 col 6 (s = 8)."""
    B = np.array(B, copy=True)
    B[:, 2] = 0.0
    B[:, 4] = B[:, 1]
    B[:, 5] = 0.5 * B[:, 0] - 2.0 * B[:, 3]
    B[:, 7] = -3.0 * B[:, 6]
    return B


def check_dependent_columns(X, tol):
    assert np.all(X[:, 2] == 0.0)
    scale = np.abs(X).max()
    assert np.abs(X[:, 4] - X[:, 1]).max() <= tol * scale
    assert np.abs(X[:, 5] - (0.5 * X[:, 0] - 2.0 * X[:, 3])).max() <= tol * scale
    assert np.abs(X[:, 7] + 3.0 * X[:, 6]).max() <= tol * scale


def _true_relres(A, B, X):
    nb = oracle.col_norms(B)
    r = oracle.col_norms(B - oracle.spmm(A, X))
    return np.where(nb > 0, r / np.where(nb > 0, nb, 1.0), 0.0)


@pytest.fixture(scope="module")
def spd():
    prob = W.problem("vardiff3d", grid=10, s=8)
    return prob.A, degenerate_block(prob.B)


@pytest.fixture(scope="module")
def nonsym():
    prob = W.problem("convdiff3d", grid=9, s=8)
    return prob.A, degenerate_block(prob.B)


@pytest.mark.parametrize("eta", [math.inf, 1e4])
@pytest.mark.parametrize("jacobi", [False, True])
def test_bcg_converges_on_rank_deficient_block(spd, eta, jacobi):
    A, B = spd
    w = oracle.jacobi_inverse_diagonal(A) if jacobi else None
    r = oracle.bcg(A, B, tol=1e-10, maxit=600, eta=eta, Minv=w, record_iterates=10)
    assert r.converged and r.status == "ok"
    assert _true_relres(A, B, r.X).max() <= 1.01e-10
    for X in r.iterates + [r.X]:
        check_dependent_columns(X, 1e-12)


def test_bcg_energy_error_no_larger_than_on_independent_columns(spd):
    A, B = spd
    Ad = A.to_dense()
    Xs = np.linalg.solve(Ad, B)
    K = 20
    full = oracle.bcg(A, B, tol=0.0, maxit=K, eta=math.inf, record_iterates=K)
    ind = oracle.bcg(A, B[:, IND], tol=0.0, maxit=K, eta=math.inf, record_iterates=K)

    def energy(E):
        return np.sqrt(np.einsum("ij,ij->j", E, Ad @ E))

    for k in range(K):
        ef = energy(full.iterates[k][:, IND] - Xs[:, IND])
        ei = energy(ind.iterates[k] - Xs[:, IND])
        assert np.all(ef <= ei * (1 + 1e-8)), (k, ef / ei)


def test_unstabilised_bcg_breaks_down_on_a_zero_column(spd):
    A, B = spd
    r = oracle.bcg(A, B, tol=1e-10, maxit=50, eta=0.0)
    assert r.status == "breakdown" and r.iters == 0 and np.all(r.X == 0.0)


def test_ir_converges_on_rank_deficient_block(spd):
    A, B = spd
    r = oracle.bcg_ir(A, B, tol=1e-10)
    assert r.converged
    assert _true_relres(A, B, r.X).max() <= 1e-10
    assert np.all(r.X[:, 2] == 0.0)
    assert np.array_equal(r.X[:, 4], r.X[:, 1])


@pytest.mark.parametrize("eta", [math.inf, 100.0])
def test_bbicgstab_converges_on_rank_deficient_block(nonsym, eta):
    A, B = nonsym
    r = oracle.bbicgstab(A, B, tol=1e-10, maxit=600, eta=eta, record_iterates=10)
    assert r.converged and r.status == "ok"
    assert _true_relres(A, B, r.X).max() <= 1.01e-10
    for X in r.iterates + [r.X]:
        check_dependent_columns(X, 1e-11)


def test_unstabilised_bbicgstab_breaks_down_on_a_zero_column(nonsym):
    A, B = nonsym
    r = oracle.bbicgstab(A, B, tol=1e-10, maxit=50, eta=0.0)
    assert r.status == "breakdown" and np.all(r.X == 0.0)


@pytest.mark.parametrize("ortho", ["mgs", "cgs2", "localized"])
def test_bgmres_converges_on_rank_deficient_block(nonsym, ortho):
    A, B = nonsym
    r = oracle.bgmres(A, B, tol=1e-10, restart=30, maxit=600, ortho=ortho, tile_rows=128)
    assert r.converged and r.status == "ok"
    assert _true_relres(A, B, r.X).max() <= 1.01e-10
    check_dependent_columns(r.X, 1e-11)
    # the tracked residual (from sigma) is the true one, zero column included
    assert np.abs(_true_relres(A, B, r.X) - r.relres).max() <= 1e-12


@pytest.mark.parametrize("ortho", ["mgs", "cgs2"])
def test_bgmres_residual_no_larger_than_on_independent_columns(nonsym, ortho):
    A, B = nonsym
    for k in (1, 3, 6, 10):
        full = oracle.bgmres(A, B, tol=0.0, restart=30, maxit=k, ortho=ortho)
        ind = oracle.bgmres(A, B[:, IND], tol=0.0, restart=30, maxit=k, ortho=ortho)
        rf = oracle.col_norms(B[:, IND] - oracle.spmm(A, full.X[:, IND]))
        ri = oracle.col_norms(B[:, IND] - oracle.spmm(A, ind.X))
        assert np.all(rf <= ri * (1 + 1e-8)), (k, rf / ri)
