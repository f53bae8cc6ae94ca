"""BBiCGStab and BGMRes(m) parity across block widths.

The FP64 row kernels are instantiated per sub-warp width (next_pow2(s) lanes
per row), so s = 1, 3, 5, 16, 32 run different code from the s = 4 and 8 of the
other tests.  12^3 convection-diffusion (1,728 rows: a ragged tail for every
row layout).  BBiCGStab: the first iterates against the oracle's within 1e-12
(k <= 5, where the oracle's own spread under a 1e-16 perturbation of B stays
below 1e-14 at every width), eta = 0 and inf, and converged solves at 1e-8.
BGMRes with CGS2 and MGS: the iterate after 1, 4, 10 and 13 Arnoldi steps
(restart 10, so 13 crosses a restart) within 1e-11, and converged solves.
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


def _op(h, prob, use):
    from paper_2104_02494_gb300.api import operator_from_problem
    return operator_from_problem(h, prob, use)


def _true_relres(prob, X):
    return oracle.col_norms(prob.B - oracle.spmm(prob.A, X)) / oracle.col_norms(prob.B)


@pytest.mark.parametrize("s", [1, 3, 5, 16, 32])
@pytest.mark.parametrize("eta", [0.0, math.inf])
def test_bbicgstab_widths(h, s, eta):
    prob = W.problem("convdiff3d", s=s, grid=12)
    op = _op(h, prob, "stencil" if s != 5 else "csr")
    ref = oracle.bbicgstab(prob.A, prob.B, tol=0.0, maxit=5, eta=eta, record_iterates=5)
    for k in (1, 2, 5):
        X, info = h.solve("bbicgstab", op, _dev(prob.B), tol=0.0, maxit=k, eta=eta)
        assert info.iters == k
        err = _rel(X.cpu().numpy(), ref.iterates[k - 1])
        assert err <= 1e-12, (k, err)
    fin = oracle.bbicgstab(prob.A, prob.B, tol=1e-8, maxit=500, eta=eta)
    X, info = h.solve("bbicgstab", op, _dev(prob.B), tol=1e-8, maxit=500, eta=eta)
    assert info.converged and fin.converged
    assert abs(info.iters - fin.iters) <= 2 + fin.iters // 10
    assert _true_relres(prob, X.cpu().numpy()).max() <= 1.5e-8
    op.close()


@pytest.mark.parametrize("s", [1, 5, 16, 32])
@pytest.mark.parametrize("ortho", ["cgs2", "mgs"])
def test_bgmres_widths(h, s, ortho):
    prob = W.problem("convdiff3d", s=s, grid=12)
    op = _op(h, prob, "stencil" if s != 5 else "csr")
    for k in (1, 4, 10, 13):
        X, info = h.solve("bgmres", op, _dev(prob.B), tol=0.0, maxit=k, restart=10, ortho=ortho)
        ref = oracle.bgmres(prob.A, prob.B, tol=0.0, restart=10, maxit=k, ortho=ortho)
        assert info.iters == k
        err = _rel(X.cpu().numpy(), ref.X)
        assert err <= 1e-11, (k, err)
    fin = oracle.bgmres(prob.A, prob.B, tol=1e-8, restart=10, maxit=400, ortho=ortho)
    X, info = h.solve("bgmres", op, _dev(prob.B), tol=1e-8, maxit=400, restart=10, ortho=ortho)
    assert info.converged and fin.converged and abs(info.iters - fin.iters) <= 1
    true = _true_relres(prob, X.cpu().numpy())
    assert true.max() <= 1.5e-8 and abs(true.max() - info.relres_max) <= 1e-10
    op.close()
