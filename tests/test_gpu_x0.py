"""GPU solvers started from a non-zero X0 (X is in/out: X0 on entry).

Every algorithm starts from R0 = B - A X0 and measures the residual relative
to ||R0_i|| (refinement: relative to ||B_i||).  Each solver's first iterates
from X0 = 0.3 N(0, 1) against the oracle's from the same X0: BCG (eta = 0, inf,
CSR and stencil), Jacobi-BCG, 1R-BCG, S_BP^p, BBiCGStab, BGMRes (CGS2, MGS,
localized), and the FP32 inner iterates of refinement; converged solves.

Unpreconditioned block CG on the log-normal diffusion field amplifies rounding
fast once the start is rough (R0 is dominated by A X0): the oracle run from X0
perturbed by 1e-16 (relative) drifts from the unperturbed one by ~3e-11 after 5
iterations and ~1e-4 after 10.  So, as for BBiCGStab elsewhere, those iterates
are compared against 100x the oracle's own measured spread (floor 1e-12), the
FP32 inner iterates against 10x the spread under a perturbation at FP32
rounding level (floor 2e-4).
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


def _x0(prob, seed=21):
    return 0.3 * W.normal_block(prob.B.shape[0], prob.B.shape[1], seed)


def _run(h, method, op, prob, X0, **kw):
    X = _dev(X0)
    X, info = h.solve(method, op, _dev(prob.B), X, **kw)
    return X.cpu().numpy(), info


def _perturbed(X0, rel, seed):
    return X0 * (1 + rel * np.random.default_rng(seed).standard_normal(X0.shape))


def _spread(run, X0, K, rel=1e-16):
    """Per iterate, the largest drift of the oracle's own run from X0 perturbed by
    ``rel`` (two draws) from its unperturbed run."""
    ref = run(X0)
    out = np.zeros(K)
    for seed in (9, 10):
        pert = run(_perturbed(X0, rel, seed))
        for k in range(K):
            out[k] = max(out[k], _rel(pert.iterates[k], ref.iterates[k]))
    return ref, out


@pytest.mark.parametrize("use", ["csr", "stencil"])
@pytest.mark.parametrize("eta", [0.0, math.inf])
def test_bcg_from_x0(h, use, eta):
    prob = W.problem("vardiff3d", grid=12, s=8)
    op = _op(h, prob, use)
    X0 = _x0(prob)
    ref, spread = _spread(lambda x: oracle.bcg(prob.A, prob.B, X0=x, tol=0.0, maxit=5, eta=eta,
                                              record_iterates=5), X0, 5)
    for k in (1, 2, 5):
        X, info = _run(h, "bcg", op, prob, X0, tol=0.0, maxit=k, eta=eta)
        err = _rel(X, ref.iterates[k - 1])
        assert info.iters == k and err <= max(1e-12, 100 * spread[k - 1]), (k, err, spread[k - 1])
        if k == 1:
            assert err <= 1e-12
    if eta == math.inf:
        fin = oracle.bcg(prob.A, prob.B, X0=X0, tol=1e-8, maxit=1000, eta=eta)
        X, info = _run(h, "bcg", op, prob, X0, tol=1e-8, maxit=1000, eta=eta)
        assert info.converged and fin.converged and abs(info.iters - fin.iters) <= 8
        n0 = oracle.col_norms(prob.B - oracle.spmm(prob.A, X0))
        assert (oracle.col_norms(prob.B - oracle.spmm(prob.A, X)) / n0).max() <= 1.5e-8
    op.close()


def test_bcg_variants_from_x0(h):
    prob = W.problem("vardiff3d", grid=12, s=8)
    op = _op(h, prob, "stencil")
    X0 = _x0(prob)
    M = h.op_jacobi(op)
    w = oracle.jacobi_inverse_diagonal(prob.A)
    cases = [(dict(precond=M), lambda x: oracle.bcg(prob.A, prob.B, X0=x, tol=0.0, maxit=10, Minv=w,
                                                   record_iterates=10)),
             (dict(one_reduction=True), lambda x: oracle.bcg_1r(prob.A, prob.B, X0=x, tol=0.0, maxit=10,
                                                               record_iterates=10)),
             (dict(p=2), lambda x: oracle.bcg(prob.A, prob.B, X0=x, tol=0.0, maxit=10, p=2,
                                             record_iterates=10))]
    for kw, run in cases:
        ref, spread = _spread(run, X0, 10)
        for k in (1, 10):
            X, info = _run(h, "bcg", op, prob, X0, tol=0.0, maxit=k, eta=math.inf, **kw)
            err = _rel(X, ref.iterates[k - 1])
            assert err <= max(1e-12, 100 * spread[k - 1]), (list(kw), k, err, spread[k - 1])
    M.close(); op.close()


@pytest.mark.parametrize("eta", [0.0, math.inf])
def test_bbicgstab_from_x0(h, eta):
    prob = W.problem("convdiff3d", grid=12, s=8)
    op = _op(h, prob, "stencil")
    X0 = _x0(prob)
    ref = oracle.bbicgstab(prob.A, prob.B, X0=X0, tol=1e-8, maxit=500, eta=eta, record_iterates=5)
    for k in (1, 2, 5):
        X, info = _run(h, "bbicgstab", op, prob, X0, tol=0.0, maxit=k, eta=eta)
        assert _rel(X, ref.iterates[k - 1]) <= 1e-12, (k, _rel(X, ref.iterates[k - 1]))
    X, info = _run(h, "bbicgstab", op, prob, X0, tol=1e-8, maxit=500, eta=eta)
    assert info.converged and ref.converged and abs(info.iters - ref.iters) <= 2
    op.close()


@pytest.mark.parametrize("ortho", ["cgs2", "mgs", "localized"])
def test_bgmres_from_x0(h, ortho):
    prob = W.problem("convdiff3d", grid=16, s=8)        # 4,096 rows: two localized tiles at s = 8
    op = _op(h, prob, "stencil")
    X0 = _x0(prob)
    for k in (1, 4, 13):
        X, info = _run(h, "bgmres", op, prob, X0, tol=0.0, maxit=k, restart=10, ortho=ortho)
        ref = oracle.bgmres(prob.A, prob.B, X0=X0, tol=0.0, restart=10, maxit=k, ortho=ortho, tile_rows=2048)
        assert _rel(X, ref.X) <= 1e-11, (k, _rel(X, ref.X))
    ref = oracle.bgmres(prob.A, prob.B, X0=X0, tol=1e-8, restart=10, maxit=400, ortho=ortho, tile_rows=2048)
    X, info = _run(h, "bgmres", op, prob, X0, tol=1e-8, restart=10, maxit=400, ortho=ortho)
    assert info.converged and ref.converged and abs(info.iters - ref.iters) <= 1
    op.close()


def test_fp32_ir_from_x0(h):
    prob = W.problem("vardiff3d", grid=12, s=8)
    op = _op(h, prob, "stencil")
    X0 = _x0(prob)
    for k in (1, 4):
        X, info = _run(h, "bcg", op, prob, X0, tol=0.0, maxit=k, prec="fp32_ir", ir_max_outer=1)
        run = lambda x: oracle.bcg_ir(prob.A, prob.B, tol=0.0, max_outer=1, inner_maxit=k, X0=x)
        ref = run(X0)
        spread = max(_rel(run(xp).X - xp, ref.X - X0)
                     for xp in (_perturbed(X0, 6e-8, 9), _perturbed(X0, 6e-8, 10)))
        err = _rel(X - X0, ref.X - X0)
        assert err <= max(2e-4, 10 * spread), (k, err, spread)
    X, info = _run(h, "bcg", op, prob, X0, tol=1e-10, maxit=5000, prec="fp32_ir")
    true = oracle.col_norms(prob.B - oracle.spmm(prob.A, X)) / oracle.col_norms(prob.B)
    assert info.converged and true.max() <= 1e-10
    op.close()
