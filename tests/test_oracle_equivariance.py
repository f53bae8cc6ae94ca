"""Pins from the algebra of block Krylov methods, independent of any one recursion.

A method in the block *-subalgebra S_B (Ch. 3.1, Def. "subalgebras") only ever
combines the columns of a block by right-multiplication with s x s matrices, so
its iterates commute with a change of basis of the right-hand sides:
X_k(B C) = X_k(B) C for every nonsingular C when the iterate is fixed by
conditions that are linear in B column by column:
  * BCG and 1R-BCG: X_k minimises the A-energy error of every column over the
    same block Krylov space span{R0 C, A R0 C, ...} = span{R0, A R0, ...}
    (Eq. "energy-minimizer"), with or without a preconditioner and for every
    re-orthonormalisation schedule (the normaliser only changes the basis);
  * BGMRes: X_k minimises every column's residual over that space (Ch. 5.1),
    whatever the orthonormalisation (MGS, CGS2, localized Arnoldi);
  * in S_BP^p the s x s quantities are block-diagonal, so the iterates commute
    only with block-diagonal C (p x p blocks); a full C breaks it;
  * BBiCGStab's omega is a single Frobenius-norm scalar (Alg.
    "BlockBiCGStab_with_reortho"), invariant under orthogonal C only.  With
    eta = 0 the blocks are the plain residuals, so the iterates commute with
    orthogonal C and not with a general one.  With eta > 0 the start block is
    normalised (R0 = R-hat sigma) and the iteration runs on the hat blocks;
    R0 C = R-hat (sigma C) and the QR of sigma C changes R-hat by an orthogonal
    factor only, so the iterates commute with every nonsingular C.
A transposed or reordered s x s product in any of the recursions breaks these.

The block GMRes iterate is also pinned directly: X_k - X_0 = V y with V an
orthonormal basis of K_k(A, R0) and y the column-wise least-squares solution of
min ||R0 - A V y|| (Ch. 5.1), computed with LAPACK on the explicit Krylov blocks.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _var7(N, seed=5, sd=1.5):
    k = np.exp(sd * np.random.default_rng(seed).standard_normal(N ** 3))
    return W.diff3d7_var(N, N, N, k)


def _convdiff():
    return W.const7(6, 5, 4, W.convdiff3d7_coeffs(6))


def _mixing(s, seed=0):
    """A well-conditioned nonsingular s x s matrix with every entry non-zero."""
    g = np.random.default_rng(seed)
    return np.eye(s) * 2.0 + 0.5 * g.standard_normal((s, s))


def _orthogonal(s, seed=0):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((s, s)))
    return Q


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("eta", [0.0, 1e4, math.inf])
@pytest.mark.parametrize("jacobi", [False, True])
def test_bcg_commutes_with_right_basis_change(eta, jacobi):
    A = _var7(5, seed=8)
    B = W.normal_block(A.n, 4, 3)
    C = _mixing(4, 1)
    w = oracle.jacobi_inverse_diagonal(A) if jacobi else None
    a = oracle.bcg(A, B, tol=0.0, maxit=6, eta=eta, Minv=w, record_iterates=6)
    b = oracle.bcg(A, B @ C, tol=0.0, maxit=6, eta=eta, Minv=w, record_iterates=6)
    for k in range(6):
        assert _rel(b.iterates[k], a.iterates[k] @ C) <= 1e-10, (k, eta, jacobi)


@pytest.mark.parametrize("eta", [0.0, math.inf])
def test_bcg_1r_commutes_with_right_basis_change(eta):
    A = _var7(5, seed=8)
    B = W.normal_block(A.n, 4, 3)
    C = _mixing(4, 2)
    a = oracle.bcg_1r(A, B, tol=0.0, maxit=6, eta=eta, record_iterates=6)
    b = oracle.bcg_1r(A, B @ C, tol=0.0, maxit=6, eta=eta, record_iterates=6)
    for k in range(6):
        assert _rel(b.iterates[k], a.iterates[k] @ C) <= 1e-10, (k, eta)


@pytest.mark.parametrize("eta", [0.0, math.inf])
def test_block_parallel_subalgebra_commutes_with_block_diagonal_change_only(eta):
    A = _var7(5, seed=8)
    s, p = 6, 2
    B = W.normal_block(A.n, s, 4)
    full = _mixing(s, 3)
    Cb = np.zeros((s, s))
    for g in range(0, s, p):
        Cb[g:g + p, g:g + p] = full[g:g + p, g:g + p]
    a = oracle.bcg(A, B, tol=0.0, maxit=5, eta=eta, p=p, record_iterates=5)
    b = oracle.bcg(A, B @ Cb, tol=0.0, maxit=5, eta=eta, p=p, record_iterates=5)
    c = oracle.bcg(A, B @ full, tol=0.0, maxit=5, eta=eta, p=p, record_iterates=5)
    for k in range(5):
        assert _rel(b.iterates[k], a.iterates[k] @ Cb) <= 1e-10, (k, eta)
    # a full change of basis mixes the groups, whose Krylov spaces differ
    assert _rel(c.iterates[4], a.iterates[4] @ full) > 1e-4


def test_bbicgstab_without_normalisation_commutes_with_orthogonal_change_only():
    A = _convdiff()
    B = W.normal_block(A.n, 4, 5)
    Q = _orthogonal(4, 6)
    C = _mixing(4, 7)
    a = oracle.bbicgstab(A, B, tol=0.0, maxit=6, eta=0.0, record_iterates=6)
    b = oracle.bbicgstab(A, B @ Q, tol=0.0, maxit=6, eta=0.0, record_iterates=6)
    c = oracle.bbicgstab(A, B @ C, tol=0.0, maxit=6, eta=0.0, record_iterates=6)
    for k in range(6):
        assert _rel(b.iterates[k], a.iterates[k] @ Q) <= 1e-10, k
    # omega = <U, S>_F / <U, U>_F of the plain residual blocks changes under a general C
    assert _rel(c.iterates[5], a.iterates[5] @ C) > 1e-6


@pytest.mark.parametrize("eta", [100.0, math.inf])
def test_normalised_bbicgstab_commutes_with_every_basis_change(eta):
    A = _convdiff()
    B = W.normal_block(A.n, 4, 5)
    C = _mixing(4, 7)
    a = oracle.bbicgstab(A, B, tol=0.0, maxit=6, eta=eta, record_iterates=6)
    c = oracle.bbicgstab(A, B @ C, tol=0.0, maxit=6, eta=eta, record_iterates=6)
    for k in range(6):
        assert _rel(c.iterates[k], a.iterates[k] @ C) <= 1e-10, (k, eta)


@pytest.mark.parametrize("ortho", ["mgs", "cgs2", "localized"])
def test_bgmres_commutes_with_right_basis_change(ortho):
    A = _convdiff()
    B = W.normal_block(A.n, 3, 8)
    C = _mixing(3, 9)
    for k in (1, 3, 7):
        a = oracle.bgmres(A, B, tol=0.0, restart=10, maxit=k, ortho=ortho, tile_rows=32)
        b = oracle.bgmres(A, B @ C, tol=0.0, restart=10, maxit=k, ortho=ortho, tile_rows=32)
        assert _rel(b.X, a.X @ C) <= 1e-10, (k, ortho)


@pytest.mark.parametrize("ortho", ["mgs", "cgs2", "localized"])
def test_bgmres_iterate_is_the_block_minimal_residual_solution(ortho):
    A = _convdiff()
    Ad = A.to_dense()
    s = 3
    B = W.normal_block(A.n, s, 10)
    X0 = 0.1 * W.normal_block(A.n, s, 11)
    R0 = B - Ad @ X0
    blocks = [R0]
    for k in range(1, 8):
        V, _ = np.linalg.qr(np.hstack(blocks))
        y, *_ = np.linalg.lstsq(Ad @ V, R0, rcond=None)
        Xk = X0 + V @ y
        r = oracle.bgmres(A, B, X0=X0, tol=0.0, restart=10, maxit=k, ortho=ortho, tile_rows=32)
        assert _rel(r.X, Xk) <= 1e-9, (k, ortho)
        blocks.append(Ad @ blocks[-1])


def test_bgmres_restart_minimises_over_the_new_space_only():
    """After a restart at m steps the space is rebuilt from the residual R_m:
    X_{m+j} = X_m + argmin over K_j(A, R_m) (restarted, not full, GMRes)."""
    A = _convdiff()
    Ad = A.to_dense()
    B = W.normal_block(A.n, 2, 12)
    m = 3
    Xm = oracle.bgmres(A, B, tol=0.0, restart=m, maxit=m).X
    Rm = B - Ad @ Xm
    blocks = [Rm]
    for j in range(1, m + 1):
        V, _ = np.linalg.qr(np.hstack(blocks))
        y, *_ = np.linalg.lstsq(Ad @ V, Rm, rcond=None)
        ref = Xm + V @ y
        got = oracle.bgmres(A, B, tol=0.0, restart=m, maxit=m + j).X
        assert _rel(got, ref) <= 1e-9, j
        blocks.append(Ad @ blocks[-1])
