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
