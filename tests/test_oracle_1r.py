"""Pins for the oracle's BCG with one reduction per iteration (Alg. "1R-CG").

The thesis states that 1R-BCG is arithmetically equivalent to Alg. "bcgaro"
(Ch. 8.1): the same iterates, with alpha^{k+1} = delta^{k+1} - beta^T alpha beta
and Q = U + Q beta replacing the product A P.  Pinned against the 2R oracle
(itself pinned elsewhere), textbook CG / PCG at s = 1, the energy minimiser over
the (preconditioned) block Krylov space and a dense direct solve; mistakes
planted in the recursion are rejected by ``test_oracle_mutations.py``.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _var7(N, seed=5, sd=1.5):
    k = np.exp(sd * np.random.default_rng(seed).standard_normal(N ** 3))
    return W.diff3d7_var(N, N, N, k)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("eta", [0.0, 1e4, math.inf])
@pytest.mark.parametrize("jacobi", [False, True])
def test_1r_equals_2r(eta, jacobi):
    """Iterate for iterate while rounding is still below the problem's own
    sensitivity: 30 iterates on the 2D Laplacian; 8 on a log-normal field,
    where 2R-BCG itself moves by 1e-4 at iteration 16 when B is perturbed by
    1e-14 (block CG's rounding divergence), so later iterates pin nothing."""
    for A, K in ((W.lap2d5(16, 15), 30), (_var7(6, sd=1.0), 8)):
        B = W.normal_block(A.n, 4, 1)
        w = oracle.jacobi_inverse_diagonal(A) if jacobi else None
        a = oracle.bcg(A, B, tol=1e-9, maxit=500, eta=eta, Minv=w, record_iterates=K)
        b = oracle.bcg_1r(A, B, tol=1e-9, maxit=500, eta=eta, Minv=w, record_iterates=K,
                          forced=a.decisions)
        assert a.converged and b.converged and abs(a.iters - b.iters) <= max(2, a.iters // 10)
        for k in range(min(K, len(a.iterates), len(b.iterates))):
            assert _rel(b.iterates[k], a.iterates[k]) <= 1e-10, (k, _rel(b.iterates[k], a.iterates[k]))
        true = oracle.col_norms(B - oracle.spmm(A, b.X)) / oracle.col_norms(B)
        assert true.max() <= 1.01e-9


def test_1r_s1_equals_textbook_cg_and_pcg():
    A = _var7(5, seed=2, sd=0.5)
    b = W.normal_block(A.n, 1, 3)
    for w in (None, oracle.jacobi_inverse_diagonal(A)):
        r = oracle.bcg_1r(A, b, tol=1e-10, maxit=300, eta=0.0, Minv=w, record_iterates=15)
        _, its, _, xs = oracle.scalar_cg(A, b[:, 0], tol=1e-10, maxit=300, record_iterates=15, minv=w)
        assert abs(r.iters - its) <= 1
        for k in range(min(15, len(xs), len(r.iterates))):
            assert _rel(r.iterates[k][:, 0], xs[k]) <= 1e-10, k


@pytest.mark.parametrize("eta", [0.0, math.inf])
def test_1r_energy_minimiser(eta):
    A = _var7(4, seed=8)
    Ad = A.to_dense()
    w = oracle.jacobi_inverse_diagonal(A)
    B = W.normal_block(A.n, 3, 4)
    r = oracle.bcg_1r(A, B, tol=0.0, maxit=4, eta=eta, Minv=w, record_iterates=4)
    blocks = [w[:, None] * B]
    for k in range(1, 5):
        V, _ = np.linalg.qr(np.hstack(blocks))
        Xk = V @ np.linalg.solve(V.T @ Ad @ V, V.T @ B)
        assert _rel(r.iterates[k - 1], Xk) <= 1e-9, k
        blocks.append(w[:, None] * (Ad @ blocks[-1]))


def test_1r_dense_solve_finite_termination():
    g = np.random.default_rng(7)
    Qm, _ = np.linalg.qr(g.standard_normal((24, 24)))
    M = (Qm * np.geomspace(1.0, 40.0, 24)) @ Qm.T
    A = W.csr_from_triples(24, *np.nonzero(np.ones((24, 24))), M.ravel())
    B = g.standard_normal((24, 4))
    r = oracle.bcg_1r(A, B, tol=1e-12, maxit=40, eta=math.inf)
    assert r.converged and r.iters <= 6 + 2
    Xs = np.linalg.solve(M, B)
    assert _rel(r.X, Xs) <= 1e-10


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_1r_replacing_every_iteration_is_the_2r_schedule(dtype):
    """With Q = A P and alpha = <P, Q> formed after every iteration (replace = 1) the
    recursion never feeds alpha or Q, so the iterates are those of Alg. "bcgaro" up to
    the rounding of the Grams (rho = <Z, R-bar> with Z a copy of R-bar here), in FP64
    and in FP32: 30 iterates on the 2D Laplacian (8 on a log-normal field, whose block
    CG amplifies rounding tenfold per iteration, as in ``test_1r_equals_2r``)."""
    for A, K in ((W.lap2d5(16, 15), 30), (_var7(6, sd=1.0), 8)):
        B = W.normal_block(A.n, 6, 3).astype(dtype)
        tol = 1e-9 if dtype == np.float64 else 1e-5
        r1 = oracle.bcg_1r(A, B, tol=tol, maxit=400, eta=math.inf, dtype=dtype, replace=1, record_iterates=K)
        r2 = oracle.bcg(A, B, tol=tol, maxit=400, eta=math.inf, dtype=dtype, record_iterates=K)
        assert r1.status == r2.status == "ok" and abs(r1.iters - r2.iters) <= max(2, r2.iters // 10)
        assert r1.replacements == r1.iters - 1
        bound = 1e-10 if dtype == np.float64 else 1e-4
        for a, b in zip(r1.iterates, r2.iterates):
            assert _rel(a, b) <= bound


def test_1r_replacement_schedule_and_fp32_breakdown():
    """replace = m forms Q and alpha directly after iterations m, 2m, ... (FP64, where the
    recursive alpha stays definite), without changing the FP64 iterates beyond rounding.
    In FP32 on the log-normal diffusion workload the plain recursion breaks down
    (alpha loses definiteness) and only replacement after every iteration converges:
    one recursive step between replacements already loses the iterates (cancellation
    in delta - beta^T alpha beta, not slow drift)."""
    A = W.lap2d5(16, 15)
    B = W.normal_block(A.n, 8, 4)
    ref = oracle.bcg(A, B, tol=1e-8, maxit=800, eta=math.inf, record_iterates=30)
    for m in (3, 7):
        r = oracle.bcg_1r(A, B, tol=1e-8, maxit=800, eta=math.inf, replace=m, record_iterates=30)
        assert r.converged and abs(r.iters - ref.iters) <= 2
        assert r.replacements == (r.iters - 1) // m
        for a, b in zip(r.iterates, ref.iterates):
            assert _rel(a, b) <= 1e-10
    prob = W.problem("vardiff3d", grid=16, s=16)
    Rs = (prob.B / oracle.col_norms(prob.B)).astype(np.float32)
    plain = oracle.bcg_1r(prob.A, Rs, tol=1e-5, maxit=300, eta=math.inf, dtype=np.float32)
    every = oracle.bcg_1r(prob.A, Rs, tol=1e-5, maxit=300, eta=math.inf, dtype=np.float32, replace=1)
    second = oracle.bcg_1r(prob.A, Rs, tol=1e-5, maxit=300, eta=math.inf, dtype=np.float32, replace=2)
    assert plain.status == "breakdown" and every.converged and not second.converged
