"""Pins for the oracle's preconditioned BCG-ARO (Alg. "bcgaro" with M != I).

The thesis's BCG finds X^k in X^0 + K_k(M^{-1} A, M^{-1} R^0) minimising the
block energy error (Ch. 4.1, Eq. "energy-minimizer"); point Jacobi takes
M = diag(A) (Ch. 2).  The pins below fix the preconditioned iteration by
means other than the oracle itself:
  * the Jacobi diagonal against the dense matrix's diagonal;
  * s = 1, eta = 0 against textbook preconditioned CG;
  * the energy minimiser over the preconditioned block Krylov space, built
    explicitly and solved by a dense Galerkin system, for eta = 0, 1e4, inf;
  * the equivalence with unpreconditioned BCG on D^{-1/2} A D^{-1/2};
  * one step to the exact solution when A is diagonal;
  * the tracked residual norms against recomputed Euclidean norms;
  * M = I given explicitly reproduces the unpreconditioned oracle exactly.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _var7(N, seed=5, sd=1.5):
    k = np.exp(sd * np.random.default_rng(seed).standard_normal(N ** 3))
    return W.diff3d7_var(N, N, N, k)


def _edge(N, seed=2):
    g = np.random.default_rng(seed)
    return W.edge2d5(N, N, np.exp(0.8 * g.standard_normal((N, N + 1))),
                     np.exp(0.8 * g.standard_normal((N + 1, N))))


def test_jacobi_inverse_diagonal_matches_dense():
    for A in (_var7(5), _edge(7), W.lap2d5(6, 4)):
        d = np.diag(A.to_dense())
        assert np.array_equal(oracle.jacobi_inverse_diagonal(A), 1.0 / d)


def test_jacobi_rejects_zero_diagonal():
    A = W.csr_from_triples(3, [0, 1, 2, 0], [0, 1, 0, 2], [2.0, 3.0, 1.0, 1.0])
    with pytest.raises(ValueError):
        oracle.jacobi_inverse_diagonal(A)


def test_pcg_s1_equals_textbook_pcg():
    A = _var7(6)
    w = oracle.jacobi_inverse_diagonal(A)
    b = W.normal_block(A.n, 1, 3)
    r = oracle.bcg(A, b, tol=1e-10, maxit=300, eta=0.0, Minv=w, record_iterates=40)
    x, its, hist, xs = oracle.scalar_cg(A, b[:, 0], tol=1e-10, maxit=300, record_iterates=40, minv=w)
    assert abs(r.iters - its) <= 1
    for k in range(min(len(xs), len(r.iterates))):
        rel = np.abs(r.iterates[k][:, 0] - xs[k]).max() / np.abs(xs[k]).max()
        assert rel <= 1e-11, (k, rel)
    # preconditioning pays on this log-normal field (sd 1.5)
    _, its0, _, _ = oracle.scalar_cg(A, b[:, 0], tol=1e-10, maxit=300)
    assert its < its0


@pytest.mark.parametrize("eta", [0.0, 1e4, math.inf])
def test_block_pcg_minimises_energy_over_preconditioned_krylov_space(eta):
    """X^k - X^0 lies in span{(M^{-1}A)^j M^{-1} R^0, j < k} and minimises
    ||X^k - X*||_{A,F}: column by column x_i = x0_i + V (V^T A V)^{-1} V^T r0_i
    with V an orthonormal basis of that span (Eq. "energy-minimizer")."""
    A = _var7(5, seed=8)
    Ad = A.to_dense()
    w = oracle.jacobi_inverse_diagonal(A)
    s = 3
    B = W.normal_block(A.n, s, 4)
    X0 = W.normal_block(A.n, s, 9) * 0.1
    r = oracle.bcg(A, B, X0=X0, tol=0.0, maxit=5, eta=eta, Minv=w, record_iterates=5)
    R0 = B - Ad @ X0
    blocks = [w[:, None] * R0]
    for k in range(1, 6):
        V, _ = np.linalg.qr(np.hstack(blocks))
        Xk = X0 + V @ np.linalg.solve(V.T @ Ad @ V, V.T @ R0)
        rel = np.abs(r.iterates[k - 1] - Xk).max() / np.abs(Xk).max()
        assert rel <= 1e-9, (k, rel)
        blocks.append(w[:, None] * (Ad @ blocks[-1]))


def test_jacobi_bcg_equals_bcg_on_symmetrically_scaled_system():
    """With M = D = diag(A): BCG on D^{-1/2} A D^{-1/2} Y = D^{-1/2} B has the
    same alpha, rho, lambda and beta, and X = D^{-1/2} Y (eta = 0)."""
    A = _edge(9)
    Ad = A.to_dense()
    d = np.diag(Ad)
    h = 1.0 / np.sqrt(d)
    As = W.csr_from_triples(A.n, *np.nonzero(Ad), (h[:, None] * Ad * h[None, :])[np.nonzero(Ad)])
    B = W.normal_block(A.n, 4, 1)
    r = oracle.bcg(A, B, tol=0.0, maxit=8, eta=0.0, Minv=1.0 / d, record_iterates=8)
    q = oracle.bcg(As, h[:, None] * B, tol=0.0, maxit=8, eta=0.0, record_iterates=8)
    for k in range(8):
        ref = h[:, None] * q.iterates[k]
        rel = np.abs(r.iterates[k] - ref).max() / np.abs(ref).max()
        assert rel <= 1e-11, (k, rel)


def test_jacobi_solves_diagonal_system_in_one_step():
    n, s = 50, 4
    d = np.geomspace(1e-3, 1e3, n)
    A = W.csr_from_triples(n, np.arange(n), np.arange(n), d)
    B = W.normal_block(n, s, 2)
    for eta in (0.0, math.inf):
        r = oracle.bcg(A, B, tol=1e-13, maxit=10, eta=eta, Minv=oracle.jacobi_inverse_diagonal(A))
        assert r.converged and r.iters == 1, (eta, r.iters)
        assert np.abs(r.X - B / d[:, None]).max() <= 1e-13 * np.abs(B / d[:, None]).max()


@pytest.mark.parametrize("eta", [0.0, 1e4, math.inf])
def test_tracked_residual_is_euclidean_with_preconditioner(eta):
    """The stopping test measures ||R_i|| (Euclidean), not the M^{-1}-norm."""
    A = _var7(6, seed=3)
    Ad = A.to_dense()
    B = W.normal_block(A.n, 5, 7)
    r = oracle.bcg(A, B, tol=1e-9, maxit=400, eta=eta, Minv=oracle.jacobi_inverse_diagonal(A))
    assert r.converged
    true = oracle.col_norms(B - Ad @ r.X) / oracle.col_norms(B)
    assert np.abs(true - r.relres).max() <= 1e-10 * max(1.0, true.max() / 1e-9)
    assert true.max() <= 1.01e-9


def test_identity_preconditioner_reproduces_unpreconditioned_oracle():
    A = _var7(5, seed=11)
    B = W.normal_block(A.n, 4, 0)
    for eta in (0.0, 1e4, math.inf):
        a = oracle.bcg(A, B, tol=1e-10, maxit=300, eta=eta)
        b = oracle.bcg(A, B, tol=1e-10, maxit=300, eta=eta, Minv=np.ones(A.n))
        assert a.iters == b.iters and a.decisions == b.decisions
        assert np.array_equal(a.X, b.X) and a.history == b.history


def test_preconditioned_float32_inner_and_refinement():
    """The FP32 iteration (dtype float32 blocks) with Jacobi, inside the
    FP64 refinement loop, still reaches FP64 accuracy."""
    A = _var7(8, seed=4)
    B = W.normal_block(A.n, 4, 5)
    w = oracle.jacobi_inverse_diagonal(A)
    ir = oracle.bcg_ir(A, B, tol=1e-12, inner_tol=1e-5, Minv=w)
    assert ir.converged
    ir0 = oracle.bcg_ir(A, B, tol=1e-12, inner_tol=1e-5)
    assert sum(ir.inner_iters) < sum(ir0.inner_iters)
