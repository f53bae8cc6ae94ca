"""Pins for the oracle's solvers: BCG-ARO, BBiCGStab-ARO, BGMRes, IR, adjoint."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _spd(n, seed, cond=50.0):
    g = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(g.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (Qm * ev) @ Qm.T


class Dense:
    """Dense matrix wrapped as CSR so that the oracle's spmm path is used."""
    def __init__(self, M):
        n = M.shape[0]
        self.n = n
        self.row_ptr = np.arange(0, n * n + 1, n, dtype=np.int32)
        self.col = np.tile(np.arange(n, dtype=np.int32), n)
        self.val = M.ravel().copy()


@pytest.mark.parametrize("n,s", [(12, 3), (30, 3), (30, 5)])
def test_bcg_reaches_direct_solve_within_ceil_n_over_s(n, s):
    M = _spd(n, n + s)
    B = np.random.default_rng(0).standard_normal((n, s))
    r = oracle.bcg(Dense(M), B, tol=1e-12, maxit=100, eta=math.inf)
    assert r.converged
    # finite termination: in exact arithmetic the residual vanishes after
    # ceil(n/s) steps; in floating point it drops by many orders there
    kstar = math.ceil(n / s)
    assert r.iters <= kstar + 2
    assert r.history[kstar - 1] <= 1e-8
    Xs = np.linalg.solve(M, B)
    assert np.abs(r.X - Xs).max() <= 1e-10 * np.abs(Xs).max()
    # residual reported from sigma equals the recomputed one
    true = oracle.col_norms(B - M @ r.X) / oracle.col_norms(B)
    assert np.abs(true - r.relres).max() < 1e-11


def test_bcg_galerkin_and_conjugacy_invariants():
    A = W.lap2d5(12, 12)
    Ad = A.to_dense()
    B = W.normal_block(A.n, 4, 0)
    r = oracle.bcg(A, B, tol=1e-14, maxit=12, eta=math.inf, record_iterates=12)
    Xs = [np.zeros_like(B)] + r.iterates
    Rs = [B - Ad @ X for X in Xs]
    D = [Xs[k + 1] - Xs[k] for k in range(len(Xs) - 1)]
    for i in range(len(Rs)):
        for j in range(i):
            c = Rs[i].T @ Rs[j]
            nrm = np.outer(oracle.col_norms(Rs[i]), oracle.col_norms(Rs[j]))
            assert np.abs(c / nrm).max() <= 1e-8
    for i in range(len(D)):
        for j in range(i):
            c = D[i].T @ Ad @ D[j]
            nrm = np.sqrt(np.outer(np.diag(D[i].T @ Ad @ D[i]), np.diag(D[j].T @ Ad @ D[j])))
            assert np.abs(c / nrm).max() <= 1e-8


def test_bcg_s1_equals_scalar_cg():
    A = W.lap3d7(6, 5, 4)
    b = W.normal_block(A.n, 1, 3)
    r = oracle.bcg(A, b, tol=1e-10, maxit=200, eta=0.0, record_iterates=60)
    x, its, hist, xs = oracle.scalar_cg(A, b[:, 0], tol=1e-10, maxit=200, record_iterates=60)
    assert abs(r.iters - its) <= 1
    K = min(len(xs), len(r.iterates))
    for k in range(K):
        rel = np.abs(r.iterates[k][:, 0] - xs[k]).max() / np.abs(xs[k]).max()
        assert rel <= 1e-12, (k, rel)


def test_parallel_subalgebra_equals_independent_scalar_cgs():
    A = W.lap2d5(10, 9)
    B = W.normal_block(A.n, 3, 4)
    r = oracle.bcg(A, B, tol=1e-9, maxit=300, eta=0.0, p=1, record_iterates=15)
    for c in range(3):
        _, its, _, xs = oracle.scalar_cg(A, B[:, c], tol=1e-9, maxit=300, record_iterates=15)
        for k in range(15):
            rel = np.abs(r.iterates[k][:, c] - xs[k]).max() / np.abs(xs[k]).max()
            assert rel <= 1e-12


@pytest.mark.parametrize("eta", [0.0, math.inf])
@pytest.mark.parametrize("s,p", [(4, 2), (6, 3), (8, 4)])
def test_block_parallel_subalgebra_equals_independent_group_solves(s, p, eta):
    """S_BP^p (Def. "subalgebras"): every s x s quantity is block diagonal, so
    the solve splits into s/p independent block-CG solves on the p-column
    groups of B, each in the block case S_B with block size p (the operator
    products are shared, the arithmetic is not)."""
    A = W.lap2d5(11, 9)
    B = W.normal_block(A.n, s, 6)
    r = oracle.bcg(A, B, tol=1e-10, maxit=200, eta=eta, p=p, record_iterates=12)
    for c0 in range(0, s, p):
        g = oracle.bcg(A, B[:, c0:c0 + p], tol=1e-10, maxit=200, eta=eta, record_iterates=12)
        for k in range(min(12, len(g.iterates), len(r.iterates))):
            ref = g.iterates[k]
            rel = np.abs(r.iterates[k][:, c0:c0 + p] - ref).max() / np.abs(ref).max()
            assert rel <= 1e-12, (c0, k, rel)


def test_bcg_chebyshev_bound():
    A = W.lap2d5(16, 16)
    Ad = A.to_dense()
    ev = np.linalg.eigvalsh(Ad)
    kappa = ev[-1] / ev[0]
    rate = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    B = W.normal_block(A.n, 4, 1)
    Xs = np.linalg.solve(Ad, B)
    r = oracle.bcg(A, B, tol=1e-12, maxit=200, eta=math.inf, record_iterates=200)
    enorm = lambda E: math.sqrt(np.sum(E * (Ad @ E)))
    e0 = enorm(Xs)
    for k, X in enumerate(r.iterates):
        assert enorm(Xs - X) <= 2 * rate ** (k + 1) * e0 * (1 + 1e-9) + 1e-12


def test_bcg_adaptive_eta_counts():
    # eta = 0: never re-orthonormalises; eta = inf: every iteration; 1e4 in between
    A = W.lap2d5(20, 20)
    B = W.normal_block(A.n, 8, 0)
    r0 = oracle.bcg(A, B, tol=1e-8, maxit=400, eta=0.0)
    ri = oracle.bcg(A, B, tol=1e-8, maxit=400, eta=math.inf)
    ra = oracle.bcg(A, B, tol=1e-8, maxit=400, eta=1e4)
    assert r0.reorths == 0 and ri.reorths == ri.iters
    assert ri.converged and ra.converged
    assert 0 <= ra.reorths <= ra.iters


def test_bcg_breakdown_on_indefinite():
    M = np.diag([1.0, -1.0, 2.0, 3.0])
    B = np.ones((4, 2))
    r = oracle.bcg(Dense(M), B, tol=1e-12, maxit=10, eta=math.inf)
    assert r.status in ("breakdown", "ok", "not_converged")
    M2 = -np.eye(4)          # negative definite: alpha is never SPD
    r2 = oracle.bcg(Dense(M2), B, tol=1e-12, maxit=10, eta=0.0)
    assert r2.status == "breakdown" and r2.iters == 0


def _textbook_bicgstab(M, b, maxit, nrec):
    x = np.zeros_like(b); r = b - M @ x; rt = r.copy(); p = r.copy()
    rho = rt @ r; xs = []
    for k in range(maxit):
        v = M @ p
        a = rho / (rt @ v)
        s_ = r - a * v
        t = M @ s_
        w = (t @ s_) / (t @ t)
        x = x + a * p + w * s_
        r = s_ - w * t
        if k < nrec:
            xs.append(x.copy())
        rho_new = rt @ r
        beta = (rho_new / rho) * (a / w)
        p = r + beta * (p - w * v)
        rho = rho_new
    return xs


def test_bbicgstab_s1_equals_textbook_and_direct_solve():
    A = W.const7(6, 5, 4, W.convdiff3d7_coeffs(5, pe=40.0))
    Ad = A.to_dense()
    assert not np.allclose(Ad, Ad.T)
    b = W.normal_block(A.n, 1, 0)
    r = oracle.bbicgstab(A, b, tol=1e-11, maxit=200, eta=0.0, record_iterates=10)
    xs = _textbook_bicgstab(Ad, b[:, 0], 10, 10)
    for k in range(min(len(xs), len(r.iterates))):
        rel = np.abs(r.iterates[k][:, 0] - xs[k]).max() / np.abs(xs[k]).max()
        assert rel <= 1e-11
    assert r.converged
    Xs = np.linalg.solve(Ad, b)
    assert np.abs(r.X - Xs).max() <= 1e-9 * np.abs(Xs).max()


@pytest.mark.parametrize("eta", [0.0, 100.0, math.inf])
def test_bbicgstab_block_converges(eta):
    A = W.const7(8, 7, 6, W.convdiff3d7_coeffs(8))
    Ad = A.to_dense()
    B = W.normal_block(A.n, 4, 0)
    r = oracle.bbicgstab(A, B, tol=1e-10, maxit=400, eta=eta)
    assert r.converged
    true = oracle.col_norms(B - Ad @ r.X) / oracle.col_norms(B)
    assert true.max() <= 1e-9
    np.testing.assert_allclose(r.X, np.linalg.solve(Ad, B), rtol=0, atol=1e-8 * np.abs(r.X).max())
    if math.isinf(eta):
        assert r.reorths == r.iters


def test_bgmres_properties():
    A = W.const7(7, 6, 5, W.convdiff3d7_coeffs(6))
    Ad = A.to_dense()
    B = W.normal_block(A.n, 3, 0)
    r = oracle.bgmres(A, B, tol=1e-10, restart=30, maxit=300)
    assert r.converged
    np.testing.assert_allclose(r.X, np.linalg.solve(Ad, B), rtol=0, atol=1e-8 * np.abs(r.X).max())
    # Frobenius residual non-increasing inside a cycle: check via truncated runs
    prev = math.inf
    for k in range(1, 12):
        rk = oracle.bgmres(A, B, tol=0.0, restart=30, maxit=k)
        R = B - Ad @ rk.X
        fro = np.linalg.norm(R)
        assert fro <= prev * (1 + 1e-12)
        prev = fro
        # per-column residual norms from sigma equal the recomputed ones
        true = oracle.col_norms(R) / oracle.col_norms(B)
        assert abs(rk.history[-1] - true.max()) <= 1e-10


def test_bgmres_exact_when_space_is_full():
    n, s = 24, 4
    g = np.random.default_rng(1)
    M = g.standard_normal((n, n)) + n * np.eye(n)
    B = g.standard_normal((n, s))
    r = oracle.bgmres(Dense(M), B, tol=1e-13, restart=n // s, maxit=n // s)
    np.testing.assert_allclose(r.X, np.linalg.solve(M, B), rtol=0, atol=1e-10)


def test_bgmres_mgs_equals_cgs2():
    A = W.const7(6, 6, 5, W.convdiff3d7_coeffs(6))
    B = W.normal_block(A.n, 4, 2)
    a = oracle.bgmres(A, B, tol=0.0, restart=10, maxit=10, ortho="mgs")
    b = oracle.bgmres(A, B, tol=0.0, restart=10, maxit=10, ortho="cgs2")
    assert np.abs(a.X - b.X).max() <= 1e-10 * np.abs(a.X).max()


def test_ir_reaches_fp64_accuracy():
    N = 8
    k = np.exp(1.5 * np.random.default_rng(1).standard_normal(N ** 3))
    A = W.diff3d7_var(N, N, N, k)
    Ad = A.to_dense()
    B = W.normal_block(A.n, 4, 0)
    r = oracle.bcg_ir(A, B, tol=1e-10, inner_tol=1e-5)
    assert r.converged
    true = oracle.col_norms(B - Ad @ r.X) / oracle.col_norms(B)
    assert true.max() <= 1e-10
    Xs = np.linalg.solve(Ad, B)
    kap = np.linalg.cond(Ad)
    assert np.abs(r.X - Xs).max() / np.abs(Xs).max() <= kap * 1e-10
    assert r.outer >= 2      # one FP32 solve alone cannot reach 1e-10
    # the FP32 inner solve alone stalls far above 1e-10
    r32 = oracle.bcg(A, B.astype(np.float32), tol=1e-12, maxit=300, dtype=np.float32)
    true32 = oracle.col_norms(B - Ad @ r32.X.astype(float)) / oracle.col_norms(B)
    assert true32.max() > 1e-9


def test_ir_from_an_initial_guess():
    """Refinement from X0: the first outer step is X0 plus the zero-start step on
    A D = B - A X0 (exactly: the same FP64 residual, the same inner solve), and
    the loop still reaches 1e-10 relative to ||B||."""
    N = 7
    k = np.exp(1.5 * np.random.default_rng(2).standard_normal(N ** 3))
    A = W.diff3d7_var(N, N, N, k)
    B = W.normal_block(A.n, 4, 3)
    X0 = 0.3 * W.normal_block(A.n, 4, 4)
    R0 = B - oracle.spmm(A, X0)
    a = oracle.bcg_ir(A, B, tol=0.0, max_outer=1, inner_maxit=6, X0=X0)
    b = oracle.bcg_ir(A, R0, tol=0.0, max_outer=1, inner_maxit=6)
    assert np.array_equal(a.X, X0 + b.X)
    r = oracle.bcg_ir(A, B, tol=1e-10, X0=X0)
    assert r.converged
    assert (oracle.col_norms(B - oracle.spmm(A, r.X)) / oracle.col_norms(B)).max() <= 1e-10


def _lap2d_eigvecs(nx, ny, modes):
    """Closed-form eigenpairs of the unscaled 5-point Dirichlet Laplacian (rows x fastest):
    v(x, y) = sin(j pi (x+1)/(nx+1)) sin(k pi (y+1)/(ny+1)),
    lambda = 4 - 2 cos(j pi/(nx+1)) - 2 cos(k pi/(ny+1))."""
    x = np.arange(nx); y = np.arange(ny)
    V, lam = [], []
    for j, k in modes:
        v = np.outer(np.sin(k * np.pi * (y + 1) / (ny + 1)), np.sin(j * np.pi * (x + 1) / (nx + 1)))
        V.append(v.ravel())
        lam.append(4 - 2 * np.cos(j * np.pi / (nx + 1)) - 2 * np.cos(k * np.pi / (ny + 1)))
    return np.array(V).T, np.array(lam)


def test_one_step_when_r0_spans_an_invariant_subspace():
    """Ch. 2 (after Thm. "cg_convergence"): a residual of grade 1 (an eigenvector) is solved in one
    iteration; in the block methods, R0 = V C with V s eigenvectors spans an A-invariant subspace,
    so X^1 = A^{-1} B = V diag(lambda)^{-1} C for BCG, 1R-BCG and BGMRes (every orthonormalisation)."""
    nx, ny = 7, 6
    A = W.lap2d5(nx, ny)
    V, lam = _lap2d_eigvecs(nx, ny, [(1, 1), (2, 3), (5, 2)])
    assert np.abs(A.to_dense() @ V - V * lam).max() <= 1e-13
    C = np.eye(3) * 2.0 + 0.5 * np.random.default_rng(3).standard_normal((3, 3))
    B = V @ C
    Xs = (V / lam) @ C
    for eta in (0.0, math.inf):
        for r in (oracle.bcg(A, B, tol=1e-12, maxit=10, eta=eta),
                  oracle.bcg_1r(A, B, tol=1e-12, maxit=10, eta=eta)):
            assert r.converged and r.iters == 1, (eta, r.iters)
            assert np.abs(r.X - Xs).max() <= 1e-12 * np.abs(Xs).max()
    for ortho in ("mgs", "cgs2", "localized"):
        r = oracle.bgmres(A, B, tol=1e-12, restart=10, maxit=10, ortho=ortho, tile_rows=16)
        assert r.converged and r.iters == 1, (ortho, r.iters)
        assert np.abs(r.X - Xs).max() <= 1e-12 * np.abs(Xs).max()
    x, its, _, _ = oracle.scalar_cg(A, V[:, 1], tol=1e-12, maxit=10)
    assert its == 1 and np.abs(x - V[:, 1] / lam[1]).max() <= 1e-12


@pytest.mark.parametrize("jacobi", [False, True])
def test_scalar_cg_reference_is_the_krylov_energy_minimiser(jacobi):
    """The textbook (P)CG used as a reference by other pins, pinned on its own: x_k minimises
    ||x - x*||_A over x0 + K_k(M^{-1}A, M^{-1}r0), built and solved densely (Ch. 2)."""
    N = 5
    k = np.exp(1.2 * np.random.default_rng(6).standard_normal(N ** 3))
    A = W.diff3d7_var(N, N, N, k)
    Ad = A.to_dense()
    w = 1.0 / np.diag(Ad) if jacobi else np.ones(A.n)
    b = W.normal_block(A.n, 1, 2)[:, 0]
    x0 = 0.1 * W.normal_block(A.n, 1, 3)[:, 0]
    x, its, hist, xs = oracle.scalar_cg(A, b, x0=x0, tol=0.0, maxit=6, record_iterates=6,
                                        minv=w if jacobi else None)
    r0 = b - Ad @ x0
    blocks = [w * r0]
    for kk in range(1, 7):
        V, _ = np.linalg.qr(np.column_stack(blocks))
        ref = x0 + V @ np.linalg.solve(V.T @ Ad @ V, V.T @ r0)
        assert np.abs(xs[kk - 1] - ref).max() <= 1e-10 * np.abs(ref).max(), kk
        blocks.append(w * (Ad @ blocks[-1]))


def test_adjoint_dense_matches_central_differences():
    nx = ny = 6; s = 3
    g = np.random.default_rng(3)
    thx = 0.5 * g.standard_normal((ny, nx + 1)); thy = 0.5 * g.standard_normal((ny + 1, nx))
    B = g.standard_normal((nx * ny, s)); Xt = g.standard_normal((nx * ny, s))

    def loss(tx, ty, Bm):
        A = W.edge2d5(nx, ny, np.exp(tx), np.exp(ty)).to_dense()
        return oracle.dense_adjoint(A, Bm, Xt)

    L, X, Lam, dA = loss(thx, thy, B)
    ax, ay = np.exp(thx), np.exp(thy)
    gx, gy = oracle.edge_theta_grad(nx, ny, ax, ay, Lam, X)
    h = 1e-6
    for (arr, gr) in ((thx, gx), (thy, gy)):
        for idx in [(0, 0), (2, 3), (ny - 1, arr.shape[1] - 1), (1, 1)]:
            p = arr.copy(); p[idx] += h
            m = arr.copy(); m[idx] -= h
            if arr is thx:
                fd = (loss(p, thy, B)[0] - loss(m, thy, B)[0]) / (2 * h)
            else:
                fd = (loss(thx, p, B)[0] - loss(thx, m, B)[0]) / (2 * h)
            assert gr[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    for idx in [(0, 0), (7, 2), (35, 1)]:
        p = B.copy(); p[idx] += h
        m = B.copy(); m[idx] -= h
        fd = (loss(thx, thy, p)[0] - loss(thx, thy, m)[0]) / (2 * h)
        assert Lam[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # scatter on the CSR pattern equals the dense dA restricted to the pattern
    Acsr = W.edge2d5(nx, ny, ax, ay)
    gsc = oracle.adjoint_scatter(Acsr, Lam, X)
    rows = np.repeat(np.arange(Acsr.n), np.diff(Acsr.row_ptr))
    np.testing.assert_allclose(gsc, dA[rows, Acsr.col], rtol=1e-13, atol=1e-13)
