"""GPU solvers on rank-deficient right-hand sides (a zero column, a duplicated
column, linear combinations), the case the residual re-orthonormalisation of
Ch. 4.3 is built for.

The normaliser completes an orthonormal basis for the deficient residual block;
which completing columns it picks is decided by rounding (duplicated columns)
or by the factorisation's tile structure (a zero column: the TSQR tiles and the
oracle's one Householder QR pick different ones).  So the iterates of the GPU
and the oracle are not comparable one by one here; what the mathematics fixes
is checked instead, against the oracle:
  * eta = 0 breaks down in the first iteration on a zero column (BCG: alpha has
    a zero row; BBiCGStab: the shadow Gram has one), with X untouched;
  * every stabilised solve converges to the tolerance; a zero column of B stays
    an exactly zero column of X; copies and combinations of columns of B give
    the same copies and combinations of X;
  * the GPU's search space contains the block Krylov space of the independent
    columns alone, so at every step each of them has an A-energy error (BCG)
    resp. residual (BGMRes) no larger than in the oracle's run on the
    independent columns alone (Eq. "energy-minimizer"; Ch. 5.1).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

from test_oracle_degenerate import IND, check_dependent_columns, degenerate_block

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


def _op(h, prob, use):
    from paper_2104_02494_gb300.api import operator_from_problem
    return operator_from_problem(h, prob, use)


def _true_relres(A, B, X):
    nb = oracle.col_norms(B)
    r = oracle.col_norms(B - oracle.spmm(A, X))
    return np.where(nb > 0, r / np.where(nb > 0, nb, 1.0), 0.0)


@pytest.fixture(scope="module")
def spd():
    prob = W.problem("vardiff3d", grid=10, s=8)
    return prob, degenerate_block(prob.B)


@pytest.fixture(scope="module")
def nonsym():
    prob = W.problem("convdiff3d", grid=16, s=8)         # 4,096 rows: two FP64 TSQR tiles at s = 8
    return prob, degenerate_block(prob.B)


@pytest.mark.parametrize("use", ["stencil", "csr"])
@pytest.mark.parametrize("eta", [math.inf, 1e4])
def test_bcg_rank_deficient(h, spd, use, eta):
    prob, B = spd
    op = _op(h, prob, use)
    ind = oracle.bcg(prob.A, B[:, IND], tol=1e-10, maxit=600, eta=eta, record_iterates=20)
    Ad = prob.A.to_dense()
    Xs = np.linalg.solve(Ad, B[:, IND])

    def energy(E):
        return np.sqrt(np.einsum("ij,ij->j", E, Ad @ E))

    for k in (1, 2, 5, 10, 20):
        X, info = h.solve("bcg", op, _dev(B), tol=0.0, maxit=k, eta=eta)
        X = X.cpu().numpy()
        assert info.iters == k
        check_dependent_columns(X, 1e-11)
        eg = energy(X[:, IND] - Xs)
        ei = energy(ind.iterates[k - 1] - Xs)
        assert np.all(eg <= ei * (1 + 1e-6)), (k, eg / ei)
    X, info = h.solve("bcg", op, _dev(B), tol=1e-10, maxit=600, eta=eta)
    X = X.cpu().numpy()
    assert info.converged and info.iters <= ind.iters + 10
    assert _true_relres(prob.A, B, X).max() <= 1.5e-10
    check_dependent_columns(X, 1e-11)
    op.close()


def test_bcg_jacobi_and_fp32_ir_rank_deficient(h, spd):
    prob, B = spd
    op = _op(h, prob, "stencil")
    M = h.op_jacobi(op)
    X, info = h.solve("bcg", op, _dev(B), tol=1e-10, maxit=600, eta=math.inf, precond=M)
    X = X.cpu().numpy()
    assert info.converged and _true_relres(prob.A, B, X).max() <= 1.5e-10
    check_dependent_columns(X, 1e-11)
    X, info = h.solve("bcg", op, _dev(B), tol=1e-10, maxit=2000, prec="fp32_ir")
    X = X.cpu().numpy()
    assert info.converged and _true_relres(prob.A, B, X).max() <= 1e-10
    assert np.all(X[:, 2] == 0.0)
    # the copies of a column may differ by the FP32 inner solves' rounding, but
    # only within the tolerance: A (X_4 - X_1) is the difference of two residuals
    d = oracle.col_norms(oracle.spmm(prob.A, X[:, [4]] - X[:, [1]]))[0]
    assert d <= 2e-10 * np.linalg.norm(B[:, 1])
    M.close(); op.close()


def test_unstabilised_solvers_break_down_on_a_zero_column(h, spd, nonsym):
    prob, B = spd
    op = _op(h, prob, "stencil")
    X, info = h.solve("bcg", op, _dev(B), tol=1e-10, maxit=50, eta=0.0)
    assert info.status == 5 and info.iters == 0 and np.all(X.cpu().numpy() == 0.0)
    op.close()
    prob, B = nonsym
    op = _op(h, prob, "stencil")
    X, info = h.solve("bbicgstab", op, _dev(B), tol=1e-10, maxit=50, eta=0.0)
    assert info.status == 5 and np.all(X.cpu().numpy() == 0.0)
    op.close()


@pytest.mark.parametrize("eta", [math.inf, 100.0])
def test_bbicgstab_rank_deficient(h, nonsym, eta):
    prob, B = nonsym
    op = _op(h, prob, "stencil")
    ref = oracle.bbicgstab(prob.A, B, tol=1e-10, maxit=600, eta=eta)
    assert ref.converged
    X, info = h.solve("bbicgstab", op, _dev(B), tol=1e-10, maxit=600, eta=eta)
    X = X.cpu().numpy()
    assert info.converged and _true_relres(prob.A, B, X).max() <= 1.5e-10
    check_dependent_columns(X, 1e-10)
    op.close()


@pytest.mark.parametrize("ortho", ["mgs", "cgs2", "localized"])
def test_bgmres_rank_deficient(h, nonsym, ortho):
    prob, B = nonsym
    op = _op(h, prob, "stencil")
    for k in (1, 3, 6, 10):
        X, info = h.solve("bgmres", op, _dev(B), tol=0.0, maxit=k, restart=30, ortho=ortho)
        X = X.cpu().numpy()
        ind = oracle.bgmres(prob.A, B[:, IND], tol=0.0, restart=30, maxit=k, ortho="mgs")
        rg = oracle.col_norms(B[:, IND] - oracle.spmm(prob.A, X[:, IND]))
        ri = oracle.col_norms(B[:, IND] - oracle.spmm(prob.A, ind.X))
        assert np.all(rg <= ri * (1 + 1e-6)), (k, rg / ri)
        check_dependent_columns(X, 1e-11)
    X, info = h.solve("bgmres", op, _dev(B), tol=1e-10, maxit=600, restart=30, ortho=ortho)
    X = X.cpu().numpy()
    true = _true_relres(prob.A, B, X)
    assert info.converged and true.max() <= 1.5e-10
    assert abs(true.max() - info.relres_max) <= 1e-11
    check_dependent_columns(X, 1e-11)
    op.close()
