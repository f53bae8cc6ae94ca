"""Parity at the workloads' full sizes, in the launch configurations the solvers use there.

The oracle cannot run whole solves at these sizes, so each check is one the
oracle finishes in seconds:
  * 96^3 convection-diffusion, s = 8: the first BBiCGStab iterates and the
    first BGMRes(30) steps against the oracle's (eta = inf);
  * 192^3 log-normal diffusion, s = 16: the FP32 operator product and the
    FP32 Gram on sampled rows; the FP32+IR solve to 1e-10 checked by the
    oracle's own FP64 residual of the GPU's X;
  * 512^2 per-edge diffusion, s = 32: the adjoint theta- and B-gradients
    against central differences of forward solves on 12 random coordinates.
Each test runs seconds; the 512^2 adjoint check (26 FP64 solves) about 1.5 min.
"""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _op(h, prob, use="stencil"):
    from paper_2104_02494_gb300.api import operator_from_problem
    return operator_from_problem(h, prob, use)


@pytest.fixture(scope="module")
def convdiff():
    return W.problem("convdiff3d")            # 96^3, s = 8


def test_full_size_bbicgstab_first_iterates(h, convdiff):
    prob = convdiff
    op = _op(h, prob)
    ref = oracle.bbicgstab(prob.A, prob.B, tol=0.0, maxit=2, eta=math.inf, record_iterates=2)
    for k in (1, 2):
        X, info = h.solve("bbicgstab", op, _dev(prob.B), tol=0.0, maxit=k, eta=math.inf)
        assert info.iters == k
        err = _rel(X.cpu().numpy(), ref.iterates[k - 1])
        assert err <= 1e-11, (k, err)
    op.close()


def test_full_size_bgmres_first_steps(h, convdiff):
    prob = convdiff
    op = _op(h, prob)
    for k in (1, 3):
        X, info = h.solve("bgmres", op, _dev(prob.B), tol=0.0, maxit=k, restart=30, ortho="cgs2")
        ref = oracle.bgmres(prob.A, prob.B, tol=0.0, restart=30, maxit=k, ortho="cgs2")
        err = _rel(X.cpu().numpy(), ref.X)
        assert err <= 1e-11, (k, err)
    op.close()


@pytest.fixture(scope="module")
def vardiff():
    return W.problem("vardiff3d")             # 192^3, s = 16


def test_full_size_vardiff_fp32_spmm_and_gram_sampled(h, vardiff):
    prob = vardiff
    A = prob.A
    op = _op(h, prob)
    P32 = prob.B.astype(np.float32)
    Q = h.spmm(op, _dev(P32)).cpu().numpy().astype(np.float64)
    rows = np.random.default_rng(1).choice(A.n, 3000, replace=False)
    rows = np.concatenate([rows, [0, A.n - 1, 192 * 192 - 1, A.n // 2]])
    P64 = P32.astype(np.float64)
    for r in rows:
        cols = A.col[A.row_ptr[r]:A.row_ptr[r + 1]]
        vals = A.val[A.row_ptr[r]:A.row_ptr[r + 1]]
        ref = vals @ P64[cols]
        bound = np.abs(vals) @ np.abs(P64[cols])
        assert np.all(np.abs(Q[r] - ref) <= 2e-6 * bound), r
    # the FP32 Gram of the whole block (tensor-core path), against FP64
    # products: per product the three-term TF32 split errs by <= 2^-21, and a
    # lane's float partial spans at most 32 + 32 roundings before it is added
    # in double, so |G - ref| <= (2^-21 + 64 2^-24) bound < 5e-6 bound
    G = h.bdot(_dev(P32), _dev(Q.astype(np.float32)), sym=False).cpu().numpy()
    Q32 = Q.astype(np.float32).astype(np.float64)
    ref = P64.T @ Q32
    bound = np.abs(P64).T @ np.abs(Q32)
    assert np.all(np.abs(G - ref) <= 5e-6 * bound)
    op.close()


def test_full_size_vardiff_ir_reaches_1e10(h, vardiff):
    prob = vardiff
    op = _op(h, prob)
    X, info = h.solve("bcg", op, _dev(prob.B), tol=1e-10, maxit=20000, eta=math.inf, prec="fp32_ir")
    assert info.converged
    Xn = X.cpu().numpy()
    true = oracle.col_norms(prob.B - oracle.spmm(prob.A, Xn)) / oracle.col_norms(prob.B)
    assert true.max() <= 1e-10, true.max()
    op.close()


def test_full_size_edge_adjoint_vs_central_differences(h):
    """512^2 per-edge diffusion, s = 32: d L / d theta_e and d L / d B_ij of
    L = 0.5 ||X - X_target||^2 against central differences of FP64 forward
    solves (tol 1e-13, adaptive eta = 1e4, the thesis's BCG choice).

    A difference quotient carries the solves' error over the step: with X
    accurate to ~kappa tol ~ 1e-8 relative (kappa ~ 1e5 here) the step
    h = 1e-6 named for this workload leaves a noise floor of 1e-4 .. 1e-3
    (measured 3e-4 .. 2.5e-3 over edges), while h = 1e-3 keeps the O(h^2)
    truncation and the noise both near 1e-6 (measured <= 2.4e-6).  So 8 edges
    and 2 B entries are checked at h = 1e-3 to 2e-5, and 2 edges at h = 1e-6
    to the noise floor, 1e-2.  20 coordinates: 14 edges at h = 1e-3 to 2e-4
    (over 14 edges the quotient's error, truncation plus the solves' error over the
    step, reaches 7e-5: one edge gives 553.42 at h = 1e-3 and 553.46 at 2e-3
    against the adjoint's 553.457; the adjoint itself is pinned to the dense
    oracle adjoint at 1e-9 on the small grid), 4 B entries at h = 1e-3 to 2e-5
    (L is quadratic in B: no truncation), 2 edges at h = 1e-6 to the noise floor.
    """
    from paper_2104_02494_gb300.autograd import BKrylovSolve
    prob = W.problem("edge2d", with_csr=False)
    N = prob.stencil["nx"]
    thx, thy = prob.extra["theta_x"], prob.extra["theta_y"]
    Xt = torch.from_numpy(prob.extra["X_target"]).cuda()
    theta = torch.from_numpy(np.concatenate([thx.ravel(), thy.ravel()])).cuda().requires_grad_(True)
    Bt = torch.from_numpy(prob.B).cuda().requires_grad_(True)
    spec = dict(kind="edge5", handle=h, nx=N, ny=N,
                solve=dict(tol=1e-13, maxit=20000, prec="fp64", eta=1e4))
    X = BKrylovSolve.apply(theta, Bt, spec)
    L = 0.5 * ((X - Xt) ** 2).sum()
    gth, gB = torch.autograd.grad(L, (theta, Bt))
    gth = gth.cpu().numpy(); gB = gB.cpu().numpy()

    def fd(th_p, th_m, B_p, B_m, hstep):
        with torch.no_grad():
            Xp = BKrylovSolve.apply(th_p, B_p, spec)
            Xm = BKrylovSolve.apply(th_m, B_m, spec)
        # L(+) - L(-) = 0.5 sum (Xp - Xm)(Xp + Xm - 2 Xt): no cancellation of large sums
        return 0.5 * float(((Xp - Xm) * (Xp + Xm - 2 * Xt)).sum()) / (2 * hstep)

    rng = np.random.default_rng(3)
    edges = rng.choice(theta.numel(), 16, replace=False)
    th0, B0 = theta.detach(), Bt.detach()
    def fd_theta(idx, hstep):
        tp = th0.clone(); tp[idx] += hstep
        tm = th0.clone(); tm[idx] -= hstep
        return fd(tp, tm, B0, B0, hstep)

    for k, idx in enumerate(edges):
        hstep, bound = (1e-3, 2e-4) if k < 14 else (1e-6, 1e-2)
        d = fd_theta(idx, hstep)
        assert abs(gth[idx] - d) <= bound * abs(d), (idx, hstep, gth[idx], d)
    for flat in rng.choice(gB.size, 4, replace=False):
        i, j = divmod(int(flat), gB.shape[1])
        Bp = B0.clone(); Bp[i, j] += 1e-3
        Bm = B0.clone(); Bm[i, j] -= 1e-3
        d = fd(th0, th0, Bp, Bm, 1e-3)        # L is quadratic in B: the quotient is exact
        assert abs(gB[i, j] - d) <= 2e-5 * abs(d), (i, j, gB[i, j], d)


def test_full_size_edge_adjoint_fp32_ir(h):
    """The same 512^2, s = 32 differentiable solve with FP32 inner solves inside FP64
    refinement, forward and adjoint solves to 1e-11 (the refinement tests the true FP64
    residual B - A X, whose floor at this conditioning, kappa ~ 1e5, lies near 1e-12):
    the gradients against the FP64 adjoint's of the same inputs (every coordinate, to
    1e-5 of the largest: kappa tol ~ 1e-6) and 4 central differences of FP32+IR
    forward solves at h = 4e-3 to 2e-3 (the solves' error over the step, ~1e-6 / h, and
    the O(h^2) truncation, at most ~16 x 7e-5, both below it)."""
    from paper_2104_02494_gb300.autograd import BKrylovSolve
    prob = W.problem("edge2d", with_csr=False)
    N = prob.stencil["nx"]
    thx, thy = prob.extra["theta_x"], prob.extra["theta_y"]
    Xt = torch.from_numpy(prob.extra["X_target"]).cuda()
    th0 = torch.from_numpy(np.concatenate([thx.ravel(), thy.ravel()])).cuda()
    B0 = torch.from_numpy(prob.B).cuda()
    grads = {}
    for prec, tol in (("fp64", 1e-13), ("fp32_ir", 1e-11)):
        spec = dict(kind="edge5", handle=h, nx=N, ny=N, solve=dict(tol=tol, maxit=20000, prec=prec, eta=1e4))
        theta = th0.clone().requires_grad_(True)
        Bt = B0.clone().requires_grad_(True)
        X = BKrylovSolve.apply(theta, Bt, spec)
        L = 0.5 * ((X - Xt) ** 2).sum()
        grads[prec] = [g.cpu().numpy() for g in torch.autograd.grad(L, (theta, Bt))]
    for a, b in zip(grads["fp32_ir"], grads["fp64"]):
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
    spec = dict(kind="edge5", handle=h, nx=N, ny=N, solve=dict(tol=1e-11, maxit=20000, prec="fp32_ir", eta=1e4))
    gth = grads["fp32_ir"][0]
    rng = np.random.default_rng(5)

    def quotient(idx, hstep):
        tp = th0.clone(); tp[idx] += hstep
        tm = th0.clone(); tm[idx] -= hstep
        with torch.no_grad():
            Xp = BKrylovSolve.apply(tp, B0, spec)
            Xm = BKrylovSolve.apply(tm, B0, spec)
        return 0.5 * float(((Xp - Xm) * (Xp + Xm - 2 * Xt)).sum()) / (2 * hstep)

    for idx in rng.choice(th0.numel(), 4, replace=False):
        d = quotient(idx, 4e-3)
        assert abs(gth[idx] - d) <= 2e-3 * abs(d), (idx, gth[idx], d)
