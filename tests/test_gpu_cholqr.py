"""FP64 BCG with the CholeskyQR2 normaliser (Def. "normalizer", Ch. 3.1; CholeskyQR2 of
Fukaya, Nakatsukasa, Yanagisawa and Yamamoto 2014) against the oracle run with the same
normaliser: iterates at 1e-12, the count of blocks that CholeskyQR2 took, its decline of
a nearly dependent block (the Householder TSQR normalises it), and the Householder mode.
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


@pytest.mark.parametrize("s", [1, 2, 5, 8, 16, 32])
def test_cholqr2_bcg_iterates(h, s):
    prob = W.problem("laplace3d", s=s, grid=16)
    op = _op(h, prob)
    ref = oracle.bcg(prob.A, prob.B, tol=1e-8, maxit=500, eta=math.inf, record_iterates=30, qr="cholqr2")
    assert ref.reorths_cholqr == ref.reorths == ref.iters
    for k in (1, 3, 10, min(30, ref.iters)):
        Xk, info = h.solve("bcg", op, _dev(prob.B), tol=0.0, maxit=k, eta=math.inf, qr="cholqr2")
        assert info.iters == k and info.reorths == k and info.reorths_cholqr == k
        assert _rel(Xk.cpu().numpy(), ref.iterates[k - 1]) <= 1e-12, (k, _rel(Xk.cpu().numpy(), ref.iterates[k - 1]))
    X, info = h.solve("bcg", op, _dev(prob.B), tol=1e-8, maxit=500, eta=math.inf, qr="cholqr2")
    assert info.converged and abs(info.iters - ref.iters) <= 2
    assert info.reorths_cholqr == info.reorths == info.iters
    true = oracle.col_norms(prob.B - oracle.spmm(prob.A, X.cpu().numpy())) / oracle.col_norms(prob.B)
    assert true.max() <= 1.5e-8
    # the Householder mode: the same solve, no CholeskyQR2 block
    Xh, ih = h.solve("bcg", op, _dev(prob.B), tol=1e-8, maxit=500, eta=math.inf, qr="householder")
    assert ih.converged and ih.reorths_cholqr == 0 and abs(ih.iters - info.iters) <= 1
    assert _rel(Xh.cpu().numpy(), X.cpu().numpy()) <= 1e-7
    op.close()


def test_cholqr2_adaptive_eta_and_jacobi(h):
    """Adaptive decisions replayed from the oracle and the point-Jacobi preconditioned
    iteration, with CholeskyQR2 on every re-orthonormalised block.  Without the
    preconditioner this workload at eta = 100 never re-orthonormalises and its iterates
    are chaotic in the rounding (the oracle's own X^k moves by 4e-12 at k = 7 when B is
    perturbed by 1e-15), so only k <= 5 is compared there."""
    prob = W.problem("vardiff3d", s=8, grid=14)
    op = _op(h, prob)
    ref = oracle.bcg(prob.A, prob.B, tol=1e-8, maxit=800, eta=100.0, record_iterates=5, qr="cholqr2")
    for k in (2, 5):
        Xk, info = h.solve("bcg", op, _dev(prob.B), tol=0.0, maxit=k, eta=100.0, forced_reortho=ref.decisions,
                           qr="cholqr2")
        assert info.reorths == sum(ref.decisions[:k]) == info.reorths_cholqr
        assert _rel(Xk.cpu().numpy(), ref.iterates[k - 1]) <= 1e-12, (k, _rel(Xk.cpu().numpy(), ref.iterates[k - 1]))
    M = h.op_jacobi(op)
    dinv = oracle.jacobi_inverse_diagonal(prob.A)
    for eta, ks in ((1e6, (5, 20, 40)), (math.inf, (1, 5, 20))):
        refm = oracle.bcg(prob.A, prob.B, tol=1e-8, maxit=800, eta=eta, Minv=dinv, record_iterates=40,
                          qr="cholqr2")
        assert refm.reorths_cholqr == refm.reorths >= 2
        for k in ks:
            Xk, info = h.solve("bcg", op, _dev(prob.B), tol=0.0, maxit=k, eta=eta, precond=M,
                               forced_reortho=refm.decisions, qr="cholqr2")
            assert info.reorths == sum(refm.decisions[:k]) == info.reorths_cholqr
            err = _rel(Xk.cpu().numpy(), refm.iterates[k - 1])
            assert err <= 1e-12, (eta, k, err)
    M.close()
    op.close()


def test_cholqr2_declines_a_nearly_dependent_block(h):
    """Columns 1 and 3 of B differ by 1e-7 relative and the first two iterations keep R
    (eta = 0, forced decisions): the block of iteration 2 has squared sines ~1e-14, the
    device declines it (below 1e-10) and the TSQR normalises; CholeskyQR2 takes the
    rest, as in the oracle, and the solution agrees with a dense solve."""
    prob = W.problem("poisson2d", s=4, grid=16)
    B = prob.B.copy()
    B[:, 3] = B[:, 1] + 1e-7 * np.linalg.norm(B[:, 1]) * prob.B[:, 3] / np.linalg.norm(prob.B[:, 3])
    forced = [False, False] + [True] * 400
    ref = oracle.bcg(prob.A, B, tol=1e-9, maxit=400, eta=0.0, forced=forced, qr="cholqr2")
    op = _op(h, prob, "csr")
    X, info = h.solve("bcg", op, _dev(B), tol=1e-9, maxit=400, eta=0.0, forced_reortho=forced, qr="cholqr2")
    # the first two iterations work with alpha of condition ~1e14 (the nearly equal
    # columns), so the rounding of any two implementations separates there and the
    # iteration counts may differ; the decline itself and the solution may not
    assert info.converged and ref.converged
    assert info.reorths_cholqr == info.reorths - 1 and ref.reorths_cholqr == ref.reorths - 1
    D = np.zeros((prob.A.n, prob.A.n))
    for i in range(prob.A.n):
        D[i, prob.A.col[prob.A.row_ptr[i]:prob.A.row_ptr[i + 1]]] = prob.A.val[prob.A.row_ptr[i]:prob.A.row_ptr[i + 1]]
    Xd = np.linalg.solve(D, B)
    assert _rel(X.cpu().numpy(), Xd) <= 1e-6
    op.close()


def test_cholqr2_rejects_unknown_qr_mode(h):
    from paper_2104_02494_gb300 import _lib as L
    prob = W.problem("poisson2d", s=2, grid=8)
    op = _op(h, prob, "csr")
    with pytest.raises(KeyError):
        h.solve("bcg", op, _dev(prob.B), qr="gram-schmidt")
    o = L.default_opts()
    assert o.qr_mode == 0
    op.close()
