"""Differentiable solve: the adjoint gradients against the oracle's dense adjoint and
against central finite differences of GPU forward solves (per-edge diffusion, a = exp(theta))."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle
    build()
    with Handle(0) as hh:
        yield hh


def _setup(N, s, seed=0):
    g = np.random.default_rng(seed)
    thx = 0.5 * g.standard_normal((N, N + 1)); thy = 0.5 * g.standard_normal((N + 1, N))
    B = g.standard_normal((N * N, s)); Xt = g.standard_normal((N * N, s))
    return thx, thy, B, Xt


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_edge_adjoint_vs_dense_and_fd(h, prec):
    from paper_2104_02494_gb300.autograd import BKrylovSolve
    N, s = 12, 3
    thx, thy, B, Xt = _setup(N, s)
    theta = torch.from_numpy(np.concatenate([thx.ravel(), thy.ravel()])).cuda().requires_grad_(True)
    Bt = torch.from_numpy(B).cuda().requires_grad_(True)
    Xtt = torch.from_numpy(Xt).cuda()
    spec = dict(kind="edge5", handle=h, nx=N, ny=N, solve=dict(tol=1e-13, maxit=3000, prec=prec))
    X = BKrylovSolve.apply(theta, Bt, spec)
    L = 0.5 * ((X - Xtt) ** 2).sum()
    gth, gB = torch.autograd.grad(L, (theta, Bt))
    gth = gth.cpu().numpy(); gB = gB.cpu().numpy()
    # oracle dense adjoint
    A = W.edge2d5(N, N, np.exp(thx), np.exp(thy)).to_dense()
    Lr, Xr, Lam, _ = oracle.dense_adjoint(A, B, Xt)
    gx, gy = oracle.edge_theta_grad(N, N, np.exp(thx), np.exp(thy), Lam, Xr)
    ref = np.concatenate([gx.ravel(), gy.ravel()])
    tol = 1e-9 if prec == "fp64" else 1e-8
    assert np.abs(gth - ref).max() <= tol * np.abs(ref).max()
    assert np.abs(gB - Lam).max() <= tol * np.abs(Lam).max()
    # central differences of GPU forward solves on a few coordinates; the step 1e-4 keeps
    # the O(h^2) truncation (~1e-8) and the solves' error over the step (~1e-13 / h) both
    # well below the bound (at h = 1e-6 the latter reaches ~1e-7 .. 1e-6)
    hstep = 1e-4
    def loss_at(th):
        with torch.no_grad():
            Xp = BKrylovSolve.apply(th, Bt.detach(), spec)
            return Xp
    rng = np.random.default_rng(3)
    for idx in rng.choice(theta.numel(), 5, replace=False):
        tp = theta.detach().clone(); tp[idx] += hstep
        tm = theta.detach().clone(); tm[idx] -= hstep
        Xp, Xm = loss_at(tp), loss_at(tm)
        # L(+) - L(-) = 0.5 sum (Xp - Xm)(Xp + Xm - 2 Xt), no cancellation of large sums
        dL = 0.5 * float(((Xp - Xm) * (Xp + Xm - 2 * Xtt)).sum())
        fd = dL / (2 * hstep)
        assert abs(gth[idx] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(ref).max()), (idx, gth[idx], fd)


def test_csr_adjoint_scatter_gradient(h):
    from paper_2104_02494_gb300.autograd import BKrylovSolve
    N, s = 10, 2
    thx, thy, B, Xt = _setup(N, s, seed=1)
    A = W.edge2d5(N, N, np.exp(thx), np.exp(thy))
    vals = torch.from_numpy(A.val.copy()).cuda().requires_grad_(True)
    spec = dict(kind="csr", handle=h, row_ptr=torch.from_numpy(A.row_ptr).cuda(),
                col=torch.from_numpy(A.col).cuda(), solve=dict(tol=1e-13, maxit=3000))
    Bt = torch.from_numpy(B).cuda()
    X = BKrylovSolve.apply(vals, Bt, spec)
    L = 0.5 * ((X - torch.from_numpy(Xt).cuda()) ** 2).sum()
    (gv,) = torch.autograd.grad(L, (vals,))
    _, Xr, Lam, dA = oracle.dense_adjoint(A.to_dense(), B, Xt)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    ref = dA[rows, A.col]
    assert np.abs(gv.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()


def test_operator_transpose(h):
    """bkrylov_op_transpose: A^T P against the oracle's product with the transposed
    matrix (integer data: bit-exact), for a non-symmetric CSR and a constant stencil."""
    from paper_2104_02494_gb300.api import operator_from_problem
    nx, ny, nz = 9, 7, 5
    c = W.convdiff3d7_coeffs(nx)
    prob = W.Problem("cd", W.const7(nx, ny, nz, c), None, dict(kind="const7", nx=nx, ny=ny, nz=nz, coeffs=c))
    At_dense = prob.A.to_dense().T
    P = np.random.default_rng(0).integers(-9, 9, (prob.A.n, 5)).astype(np.float64)
    for use in ("csr", "stencil"):
        op = operator_from_problem(h, prob, use)
        opT = h.op_transpose(op)
        Q = h.spmm(opT, torch.from_numpy(P).cuda()).cpu().numpy()
        ref = At_dense @ P
        assert np.abs(Q - ref).max() <= 1e-13 * np.abs(At_dense).sum(axis=1).max() * 9, use
        opT.close(); op.close()
    # integer CSR values: exact
    A = W.csr_from_triples(4, [0, 0, 1, 2, 3, 3, 1], [0, 2, 1, 3, 0, 3, 0], [2.0, -1.0, 3.0, 5.0, -4.0, 1.0, 7.0])
    op = h.op_csr(torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col).cuda(), torch.from_numpy(A.val).cuda())
    opT = h.op_transpose(op)
    P = np.arange(8, dtype=np.float64).reshape(4, 2) - 3
    assert np.array_equal(h.spmm(opT, torch.from_numpy(P).cuda()).cpu().numpy(), A.to_dense().T @ P)
    opT.close(); op.close()


@pytest.mark.parametrize("method", ["bbicgstab", "bgmres"])
def test_csr_adjoint_nonsymmetric(h, method):
    """A non-symmetric CSR (upwind convection-diffusion): the adjoint solve runs on A^T,
    checked against the oracle's dense adjoint (Lambda = A^{-T} (X - X_target))."""
    from paper_2104_02494_gb300.autograd import BKrylovSolve
    N, s = 6, 3
    c = W.convdiff3d7_coeffs(N)
    A = W.const7(N, N, N, c)
    g = np.random.default_rng(4)
    B = g.standard_normal((A.n, s)); Xt = g.standard_normal((A.n, s))
    vals = torch.from_numpy(A.val.copy()).cuda().requires_grad_(True)
    solve = dict(tol=1e-13, maxit=3000) if method == "bbicgstab" else dict(tol=1e-13, maxit=3000, restart=40)
    spec = dict(kind="csr", handle=h, method=method, row_ptr=torch.from_numpy(A.row_ptr).cuda(),
                col=torch.from_numpy(A.col).cuda(), solve=solve)
    Bt = torch.from_numpy(B).cuda().requires_grad_(True)
    X = BKrylovSolve.apply(vals, Bt, spec)
    L = 0.5 * ((X - torch.from_numpy(Xt).cuda()) ** 2).sum()
    gv, gB = torch.autograd.grad(L, (vals, Bt))
    _, Xr, Lam, dA = oracle.dense_adjoint(A.to_dense(), B, Xt)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    ref = dA[rows, A.col]
    assert np.abs(gB.cpu().numpy() - Lam).max() <= 1e-9 * np.abs(Lam).max()
    assert np.abs(gv.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()


def test_autograd_releases_operators(h):
    """No operator outlives a forward or backward: no_grad forwards, a backward that never
    runs and a second backward (retain_graph) leave the handle's operators and the device
    memory in use where they were."""
    from paper_2104_02494_gb300.autograd import BKrylovSolve
    N, s = 16, 2
    thx, thy, B, Xt = _setup(N, s, seed=2)
    theta = torch.from_numpy(np.concatenate([thx.ravel(), thy.ravel()])).cuda().requires_grad_(True)
    Bt = torch.from_numpy(B).cuda()
    spec = dict(kind="edge5", handle=h, nx=N, ny=N, solve=dict(tol=1e-12, maxit=3000))
    BKrylovSolve.apply(theta.detach(), Bt, spec)     # warm-up: workspace grown once
    torch.cuda.synchronize()
    n_ops, mem = len(h._ops), torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    with torch.no_grad():
        for _ in range(5):
            BKrylovSolve.apply(theta, Bt, spec)
    X = BKrylovSolve.apply(theta, Bt, spec)           # graph built, backward never run
    del X
    X = BKrylovSolve.apply(theta, Bt, spec)
    L = ((X - torch.from_numpy(Xt).cuda()) ** 2).sum()
    g1 = torch.autograd.grad(L, theta, retain_graph=True)[0]
    g2 = torch.autograd.grad(L, theta)[0]
    assert torch.equal(g1, g2)
    del X, L, g1, g2
    torch.cuda.synchronize()
    assert len(h._ops) == n_ops
    assert torch.cuda.memory_allocated() == mem
    assert torch.cuda.mem_get_info()[0] == free0
