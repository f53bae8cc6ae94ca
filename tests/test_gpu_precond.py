"""GPU parity of the preconditioned BCG-ARO (Alg. "bcgaro" with M = point Jacobi).

  * the Jacobi diagonal diag(A)^{-1} of every operator kind against the
    oracle's (bit-exact for CSR and the constant stencil, 2 ulp for the
    stencils whose diagonal the library sums itself), and the FP32 diagonal
    operator bit-exact;
  * FP64 iterates X^k (k <= 20) against the oracle's preconditioned BCG to
    1e-12, for eta = 0, inf and the oracle's replayed adaptive schedule, on
    CSR and matrix-free operators, s in {1, 4, 8, 16, 32}, and in S_BP^p;
  * the FP32 inner iterates against the oracle's float32 BCG (2e-4, as for
    the unpreconditioned FP32 path) and the FP32+IR solve to 1e-10;
  * converged solves: Euclidean residual <= tol (the stopping test does not
    use the M^{-1}-norm), iteration counts within 2 of the oracle's;
  * graph replay against direct launches, and the error paths.
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


def _jacobi(h, op):
    M = h.op_jacobi(op)
    w = h.spmm(M, torch.ones(op.n, 1, dtype=torch.float64, device="cuda")).cpu().numpy()[:, 0]
    return M, w


@pytest.mark.parametrize("name,grid,use", [("vardiff3d", 10, "csr"), ("vardiff3d", 10, "stencil"),
                                           ("edge2d", 24, "csr"), ("edge2d", 24, "stencil"),
                                           ("convdiff3d", 9, "stencil"), ("poisson2d", 16, "csr")])
def test_jacobi_diagonal(h, name, grid, use):
    prob = W.problem(name, grid=grid)
    op = _op(h, prob, use)
    M, w = _jacobi(h, op)
    ref = oracle.jacobi_inverse_diagonal(prob.A)
    if use == "csr" or prob.stencil["kind"] == "const7":
        assert np.array_equal(w, ref)
    else:
        assert np.all(np.abs(w - ref) <= 4.5e-16 * np.abs(ref))
    # the diagonal operator in FP32: row i times float(w_i), one IEEE product
    P = np.random.default_rng(0).standard_normal((op.n, 8)).astype(np.float32)
    Q = h.spmm(M, _dev(P)).cpu().numpy()
    assert np.array_equal(Q, w.astype(np.float32)[:, None] * P)
    M.close(); op.close()


def test_jacobi_and_diag_errors(h):
    from paper_2104_02494_gb300.api import BkError
    A = W.csr_from_triples(3, [0, 1, 2, 0], [0, 1, 0, 2], [2.0, 3.0, 1.0, 1.0])   # a_22 = 0
    dv = lambda a: torch.from_numpy(np.asarray(a)).cuda()
    op = h.op_csr(dv(A.row_ptr), dv(A.col), dv(A.val))
    with pytest.raises(BkError):
        h.op_jacobi(op)
    op.close()
    prob = W.problem("poisson2d", grid=16)
    op = _op(h, prob, "stencil")
    M = h.op_diag(torch.ones(op.n + 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(BkError):                      # n differs from A's
        h.solve("bcg", op, _dev(prob.B), tol=1e-8, maxit=10, precond=M)
    M.close()
    M = h.op_jacobi(op)
    for method in ("bbicgstab", "bgmres"):            # BCG only
        with pytest.raises(BkError):
            h.solve(method, op, _dev(prob.B), tol=1e-8, maxit=10, precond=M)
    M.close(); op.close()


@pytest.mark.parametrize("eta", [0.0, math.inf])
@pytest.mark.parametrize("name,grid,s,use", [("vardiff3d", 12, 8, "stencil"), ("vardiff3d", 12, 4, "csr"),
                                             ("edge2d", 32, 32, "stencil"), ("edge2d", 32, 16, "csr"),
                                             ("vardiff3d", 12, 1, "stencil")])
def test_pcg_fp64_iterates_and_final(h, name, grid, s, use, eta):
    prob = W.problem(name, grid=grid, s=s)
    op = _op(h, prob, use)
    M, w = _jacobi(h, op)
    wref = oracle.jacobi_inverse_diagonal(prob.A)
    ref = oracle.bcg(prob.A, prob.B, tol=1e-8, maxit=2000, eta=eta, Minv=wref, record_iterates=20)
    for k in (1, 2, 5, 20):
        X, info = h.solve("bcg", op, _dev(prob.B), tol=0.0, maxit=k, eta=eta, precond=M)
        assert info.iters == k
        err = _rel(X.cpu().numpy(), ref.iterates[k - 1])
        assert err <= 1e-12, (k, err)
    X, info = h.solve("bcg", op, _dev(prob.B), tol=1e-8, maxit=2000, eta=eta, precond=M)
    assert info.converged and ref.converged and abs(info.iters - ref.iters) <= 2
    true = oracle.col_norms(prob.B - oracle.spmm(prob.A, X.cpu().numpy())) / oracle.col_norms(prob.B)
    assert true.max() <= 1.5e-8
    assert abs(true.max() - info.relres_max) <= 1e-3 * true.max() + 1e-12
    M.close(); op.close()


def test_pcg_adaptive_eta_with_replay(h):
    prob = W.problem("vardiff3d", grid=14, s=8)
    op = _op(h, prob, "stencil")
    M, _ = _jacobi(h, op)
    wref = oracle.jacobi_inverse_diagonal(prob.A)
    ref = oracle.bcg(prob.A, prob.B, tol=1e-8, maxit=500, eta=1e4, Minv=wref, record_iterates=30)
    X, info = h.solve("bcg", op, _dev(prob.B), tol=1e-8, maxit=500, eta=1e4, precond=M)
    assert info.converged
    K = min(len(info.decisions), len(ref.decisions))
    assert sum(a != b for a, b in zip(info.decisions[:K], ref.decisions[:K])) <= 2
    for k in (5, 30):
        X, _ = h.solve("bcg", op, _dev(prob.B), tol=0.0, maxit=k, eta=1e4, precond=M,
                       forced_reortho=ref.decisions)
        assert _rel(X.cpu().numpy(), ref.iterates[k - 1]) <= 1e-12
    M.close(); op.close()


@pytest.mark.parametrize("s,p", [(8, 2), (8, 4), (12, 4)])
def test_pcg_block_parallel_subalgebra(h, s, p):
    prob = W.problem("vardiff3d", grid=12, s=s)
    op = _op(h, prob, "stencil")
    M, _ = _jacobi(h, op)
    wref = oracle.jacobi_inverse_diagonal(prob.A)
    for eta in (0.0, math.inf):
        ref = oracle.bcg(prob.A, prob.B, tol=0.0, maxit=10, eta=eta, p=p, Minv=wref, record_iterates=10)
        for k in (1, 10):
            X, _ = h.solve("bcg", op, _dev(prob.B), tol=0.0, maxit=k, eta=eta, p=p, precond=M)
            assert _rel(X.cpu().numpy(), ref.iterates[k - 1]) <= 1e-12, (eta, k)
    M.close(); op.close()


@pytest.mark.parametrize("s", [4, 6, 16, 32])
@pytest.mark.parametrize("eta", [math.inf, 0.0])
def test_pcg_fp32_inner_iterates(h, s, eta):
    prob = W.problem("vardiff3d", s=s, grid=12)
    op = _op(h, prob, "stencil")
    M, _ = _jacobi(h, op)
    wref = oracle.jacobi_inverse_diagonal(prob.A)
    for k in (1, 2, 4):
        X, info = h.solve("bcg", op, _dev(prob.B), tol=0.0, maxit=k, eta=eta, prec="fp32_ir",
                          ir_max_outer=1, precond=M)
        ref = oracle.bcg_ir(prob.A, prob.B, tol=0.0, max_outer=1, inner_maxit=k, eta=eta, Minv=wref)
        assert info.iters == k and ref.inner_iters == [k]
        assert _rel(X.cpu().numpy(), ref.X) <= 2e-4, (s, eta, k, _rel(X.cpu().numpy(), ref.X))
    M.close(); op.close()


def test_pcg_fp32_ir_reaches_1e10_with_fewer_inner_iterations(h):
    prob = W.problem("vardiff3d", s=16, grid=20)
    op = _op(h, prob, "stencil")
    M, _ = _jacobi(h, op)
    X, info = h.solve("bcg", op, _dev(prob.B), tol=1e-10, maxit=5000, prec="fp32_ir", precond=M)
    true = oracle.col_norms(prob.B - oracle.spmm(prob.A, X.cpu().numpy())) / oracle.col_norms(prob.B)
    assert info.converged and true.max() <= 1e-10
    X0, info0 = h.solve("bcg", op, _dev(prob.B), tol=1e-10, maxit=5000, prec="fp32_ir")
    assert info0.converged and info.iters < info0.iters
    M.close(); op.close()


def test_pcg_graph_replay_equals_direct_launches(h):
    prob = W.problem("vardiff3d", grid=16, s=4)
    op = _op(h, prob, "csr")
    M, _ = _jacobi(h, op)
    Xg, ig = h.solve("bcg", op, _dev(prob.B), tol=1e-8, maxit=1000, precond=M)
    Xd, idr = h.solve("bcg", op, _dev(prob.B), tol=1e-8, maxit=1000, precond=M, profile=True)
    assert ig.iters == idr.iters and ig.iters > 40
    assert np.array_equal(Xg.cpu().numpy(), Xd.cpu().numpy())
    launches = {p[0]: p[2] for p in h.profile()}
    assert launches["precond_rho"] >= idr.iters
    M.close(); op.close()


@pytest.mark.parametrize("n,s", [(100003, 16), (65537, 32), (777, 16), (3, 32)])
def test_diag_pass_fp32_stream(h, n, s):
    """The FP32 diagonal pass (Z = diag(w) X with rho = X^T Z, the preconditioner step of the
    inner solves) on ragged row counts: Z bit-exact (one IEEE product per entry), rho within
    the FP32 Gram bound of the other Gram tests."""
    g = np.random.default_rng(n + s)
    w = np.exp(g.standard_normal(n))
    M = h.op_diag(torch.from_numpy(w).cuda())
    P = g.standard_normal((n, s)).astype(np.float32)
    Z, G = h.spmm_gram(M, _dev(P), sym=True)
    w32 = w.astype(np.float32)
    assert np.array_equal(Z.cpu().numpy(), w32[:, None] * P)
    P64 = P.astype(np.float64)
    Z64 = (w32[:, None] * P).astype(np.float64)
    Gref = P64.T @ Z64
    bound = np.abs(P64).T @ np.abs(Z64)
    assert np.all(np.abs(G.cpu().numpy() - Gref) <= (2.0 ** -21 + 64 * 2.0 ** -24) * bound + 1e-30)
    M.close()
