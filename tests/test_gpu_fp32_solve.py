"""The raw FP32 block CG solve, FP32 CSR values and the Frobenius stopping measure.

Raw FP32 BCG (Alg. "bcgaro" with FP32 blocks and products and every s x s
quantity in FP64, the thesis's single-precision runs of Ch. 4.4):
  * its first iterates within 2e-4 (max-norm relative) of the oracle's float32
    BCG on the same input (both carry FP32 rounding; the bound is the one of the
    FP32 inner-solve parity tests);
  * solved to tol = 1e-5, the relative residual recomputed by the oracle in
    FP64 is at most 1.5e-5 in every column (the recursively tracked FP32
    residual drifts from the true one by O(eps_32 kappa)), and the error
    against the oracle's FP64 solution is reported.
FP32 CSR values: an operator built from float values is the same matrix in both
precisions (bitwise the results of the operator built from their exact FP64
widening).  Frobenius measure (norm="fro", reading c2): the GPU solvers stop
within one iteration of the oracle's Frobenius run, and the true residual meets
the tolerance in that norm.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle.blockops import spmm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle
    build()
    with Handle(0) as hh:
        yield hh


def _op(h, prob, use):
    from paper_2104_02494_gb300.api import operator_from_problem
    return operator_from_problem(h, prob, use)


def _true_relres(A, B, X):
    R = B - spmm(A, X.astype(np.float64))
    return np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)


@pytest.mark.parametrize("use", ["csr", "stencil"])
def test_raw_fp32_first_iterates(h, use):
    prob = W.problem("poisson2d", s=4, grid=40)
    op = _op(h, prob, use)
    B32 = prob.B.astype(np.float32)
    ref = oracle.bcg(prob.A, B32, tol=0.0, maxit=6, eta=math.inf, dtype=np.float32, record_iterates=6)
    Bd = torch.from_numpy(B32).cuda()
    for k in range(1, 7):
        X, info = h.solve("bcg", op, Bd, tol=0.0, maxit=k, eta=math.inf, prec="fp32")
        Xk = X.cpu().numpy().astype(np.float64)
        Rk = ref.iterates[k - 1].astype(np.float64)
        err = np.abs(Xk - Rk).max() / np.abs(Rk).max()
        assert info.iters == k and err <= 2e-4, (use, k, err)
    op.close()


@pytest.mark.parametrize("case", ["poisson2d-csr", "laplace3d-stencil", "vardiff3d-jacobi"])
def test_raw_fp32_solve_to_1e5(h, case):
    name, use = case.split("-")
    if name == "poisson2d":
        prob = W.problem("poisson2d", s=4)
    elif name == "laplace3d":
        prob = W.problem("laplace3d", s=8, grid=32)
    else:
        prob = W.problem("vardiff3d", s=16, grid=20)
    op = _op(h, prob, "stencil" if use != "csr" else "csr")
    M = h.op_jacobi(op) if use == "jacobi" else None
    Bd = torch.from_numpy(prob.B.astype(np.float32)).cuda()
    X, info = h.solve("bcg", op, Bd, tol=1e-5, maxit=5000, eta=math.inf, prec="fp32", precond=M)
    assert info.converged, info
    X64 = X.cpu().numpy().astype(np.float64)
    rel = _true_relres(prob.A, prob.B, X64)
    Xs = oracle.bcg(prob.A, prob.B, tol=1e-12, maxit=20000, eta=0.0,
                    Minv=oracle.jacobi_inverse_diagonal(prob.A)).X
    err = np.linalg.norm(X64 - Xs) / np.linalg.norm(Xs)
    print(f"raw FP32 {case}: iters {info.iters}, true relres max {rel.max():.3e}, "
          f"error vs FP64 solution {err:.3e}")
    assert rel.max() <= 1.5e-5, (case, rel.max())
    if M is not None:
        M.close()
    op.close()


def test_fp32_csr_values_same_matrix(h):
    prob = W.problem("vardiff3d", s=8, grid=12)
    A = prob.A
    v32 = A.val.astype(np.float32)
    rp = torch.from_numpy(A.row_ptr.astype(np.int32)).cuda()
    cl = torch.from_numpy(A.col.astype(np.int32)).cuda()
    op32 = h.op_csr(rp, cl, torch.from_numpy(v32).cuda())
    op64 = h.op_csr(rp, cl, torch.from_numpy(v32.astype(np.float64)).cuda())
    B = torch.from_numpy(prob.B).cuda()
    X1, i1 = h.solve("bcg", op32, B, tol=1e-10, maxit=2000)
    X2, i2 = h.solve("bcg", op64, B, tol=1e-10, maxit=2000)
    assert i1.iters == i2.iters and torch.equal(X1, X2)
    P = torch.randn(A.n, 8, device="cuda", dtype=torch.float32)
    assert torch.equal(h.spmm(op32, P), h.spmm(op64, P))
    Y1, _ = h.solve("bcg", op32, B, tol=1e-10, maxit=50, prec="fp32_ir")
    Y2, _ = h.solve("bcg", op64, B, tol=1e-10, maxit=50, prec="fp32_ir")
    assert torch.equal(Y1, Y2)
    op32.close(); op64.close()


@pytest.mark.parametrize("method", ["bcg", "bbicgstab", "bgmres", "bcg_fp32_ir"])
def test_frobenius_stopping(h, method):
    if method == "bcg":
        prob = W.problem("poisson2d", s=4, grid=30)
        kw = dict(eta=math.inf)
        ref = oracle.bcg(prob.A, prob.B, tol=1e-8, eta=math.inf, norm="fro")
    elif method == "bbicgstab":
        prob = W.problem("convdiff3d", s=3, grid=10)
        kw = dict(eta=100.0)
        ref = oracle.bbicgstab(prob.A, prob.B, tol=1e-8, eta=100.0, norm="fro")
    elif method == "bgmres":
        prob = W.problem("convdiff3d", s=3, grid=10)
        kw = dict(restart=10, ortho="mgs")
        ref = oracle.bgmres(prob.A, prob.B, tol=1e-8, restart=10, ortho="mgs", norm="fro")
    else:
        prob = W.problem("vardiff3d", s=4, grid=10)
        kw = dict(eta=math.inf, prec="fp32_ir")
        ref = oracle.bcg_ir(prob.A, prob.B, tol=1e-10, norm="fro")
    op = _op(h, prob, "csr")
    tol = 1e-10 if method == "bcg_fp32_ir" else 1e-8
    X, info = h.solve(method.split("_")[0], op, torch.from_numpy(prob.B).cuda(), tol=tol, maxit=5000,
                      norm="fro", **kw)
    assert info.converged
    Xh = X.cpu().numpy()
    fro = np.linalg.norm(prob.B - spmm(prob.A, Xh)) / np.linalg.norm(prob.B)
    assert fro <= tol * 1.05, (method, fro)
    if method == "bcg_fp32_ir":
        assert abs(info.outer - ref.outer) <= 1
    else:
        assert abs(info.iters - ref.iters) <= 1, (method, info.iters, ref.iters)
        Xm, im = h.solve(method, op, torch.from_numpy(prob.B).cuda(), tol=tol, maxit=5000, norm="max", **kw)
        assert info.iters <= im.iters
    op.close()
