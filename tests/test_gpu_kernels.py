"""GPU kernel parity against the oracle: BOP (CSR + stencils), BDOT, TSQR, adjoint kernels.

Every call goes through the C ABI (ctypes binding); the oracle runs on the
CPU on the same seeded inputs.  Tolerances:
  * integer-valued inputs: bit-exact (every product and partial sum is an
    exactly representable integer, so summation order cannot matter);
  * FP64 random inputs: 1e-13 relative to the magnitude bound of each entry
    (a few ulps times the number of terms);
  * FP32: 2e-6 relative to the magnitude bound.
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


def _ops(h, grid=(9, 7, 5)):
    """(name, CSR oracle matrix, GPU operator) for every operator kind."""
    from paper_2104_02494_gb300.api import operator_from_problem
    nx, ny, nz = grid
    out = []
    lap = W.problem("laplace3d", s=1, grid=1)
    lap.A = W.lap3d7(nx, ny, nz)
    lap.stencil = dict(kind="const7", nx=nx, ny=ny, nz=nz, coeffs=W.LAPL7)
    out.append(("lap7-csr", lap.A, operator_from_problem(h, lap, "csr")))
    out.append(("lap7-stencil", lap.A, operator_from_problem(h, lap, "stencil")))
    c = W.convdiff3d7_coeffs(nx)
    cd = W.Problem("cd", W.const7(nx, ny, nz, c), None, dict(kind="const7", nx=nx, ny=ny, nz=nz, coeffs=c))
    out.append(("convdiff-stencil", cd.A, operator_from_problem(h, cd, "stencil")))
    k = np.exp(1.5 * np.random.default_rng(1).standard_normal(nx * ny * nz))
    vd = W.Problem("vd", W.diff3d7_var(nx, ny, nz, k), None, dict(kind="var7", nx=nx, ny=ny, nz=nz, k=k))
    out.append(("var7-stencil", vd.A, operator_from_problem(h, vd, "stencil")))
    out.append(("var7-csr", vd.A, operator_from_problem(h, vd, "csr")))
    g = np.random.default_rng(2)
    ax = np.exp(0.5 * g.standard_normal((ny, nx + 1))); ay = np.exp(0.5 * g.standard_normal((ny + 1, nx)))
    ed = W.Problem("ed", W.edge2d5(nx, ny, ax, ay), None, dict(kind="edge5", nx=nx, ny=ny, nz=1, ax=ax, ay=ay))
    out.append(("edge5-stencil", ed.A, operator_from_problem(h, ed, "stencil")))
    out.append(("edge5-csr", ed.A, operator_from_problem(h, ed, "csr")))
    return out


def _absbound(A, P):
    """|A| |P| entrywise: the magnitude scale of each output of A P."""
    Aabs = W.CSR(A.n, A.row_ptr, A.col, np.abs(A.val))
    return oracle.spmm(Aabs, np.abs(P))


@pytest.mark.parametrize("s", [1, 3, 4, 8, 16, 32])
def test_spmm_fp64_all_operators(h, s):
    for name, A, op in _ops(h):
        P = np.random.default_rng(s).standard_normal((A.n, s))
        Q = h.spmm(op, _dev(P)).cpu().numpy()
        ref = oracle.spmm(A, P)
        err = np.abs(Q - ref) / (_absbound(A, P) + 1e-300)
        assert err.max() <= 1e-14, (name, s, err.max())


def test_spmm_integer_inputs_bit_exact(h):
    for s in (1, 5, 8, 32):
        for name, A, op in _ops(h, grid=(17, 11, 6))[:2]:     # integer Laplacian (CSR, stencil)
            P = np.random.default_rng(s).integers(-1000, 1000, (A.n, s)).astype(np.float64)
            Q = h.spmm(op, _dev(P)).cpu().numpy()
            assert np.array_equal(Q, oracle.spmm(A, P)), (name, s)


@pytest.mark.parametrize("s", [1, 4, 16, 32])
def test_spmm_fp32(h, s):
    for name, A, op in _ops(h):
        P = np.random.default_rng(s).standard_normal((A.n, s)).astype(np.float32)
        Q = h.spmm(op, _dev(P)).cpu().numpy().astype(np.float64)
        ref = oracle.spmm(A, P.astype(np.float64))
        err = np.abs(Q - ref) / (_absbound(A, P.astype(np.float64)) + 1e-30)
        assert err.max() <= 2e-6, (name, s, err.max())


def test_residual_kernel(h):
    for name, A, op in _ops(h)[:3]:
        g = np.random.default_rng(0)
        B = g.standard_normal((A.n, 6)); X = g.standard_normal((A.n, 6))
        R = h.residual(op, _dev(B), _dev(X)).cpu().numpy()
        ref = B - oracle.spmm(A, X)
        assert np.abs(R - ref).max() <= 1e-13 * (np.abs(B).max() + _absbound(A, X).max())


@pytest.mark.parametrize("n", [1, 37, 1000, 100003])
@pytest.mark.parametrize("s", [1, 2, 7, 8, 32])
def test_bdot_fp64(h, n, s):
    g = np.random.default_rng(n + s)
    X = g.standard_normal((n, s)); Y = g.standard_normal((n, s))
    bound = np.abs(X).T @ np.abs(Y)
    for sym in (False, True):
        G = h.bdot(_dev(X), _dev(Y), sym=sym).cpu().numpy()
        ref = oracle.gram(X, Y, sym=sym)
        assert np.all(np.abs(G - ref) <= 1e-13 * (bound + bound.T) + 1e-300), (n, s, sym)
    # symmetric Gram of a block with itself is exactly symmetric
    G = h.bdot(_dev(X), _dev(X), sym=True).cpu().numpy()
    assert np.array_equal(G, G.T)


def test_bdot_integer_bit_exact_and_deterministic(h):
    g = np.random.default_rng(3)
    X = g.integers(-20, 20, (54321, 9)).astype(np.float64)
    Y = g.integers(-20, 20, (54321, 9)).astype(np.float64)
    G1 = h.bdot(_dev(X), _dev(Y)).cpu().numpy()
    assert np.array_equal(G1, X.T @ Y)
    Xr, Yr = _dev(g.standard_normal((77777, 16))), _dev(g.standard_normal((77777, 16)))
    a = h.bdot(Xr, Yr).cpu().numpy(); b = h.bdot(Xr, Yr).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [1, 37, 40000, 300007])
@pytest.mark.parametrize("s", [3, 4, 8, 12, 16, 32])
def test_bdot_fp32(h, n, s):
    # s % 4 == 0 runs the vectorised (float4) layout, other widths the scalar one
    g = np.random.default_rng(4 + n + s)
    X = g.standard_normal((n, s)).astype(np.float32); Y = g.standard_normal((n, s)).astype(np.float32)
    ref = X.astype(np.float64).T @ Y.astype(np.float64)
    bound = np.abs(X.astype(np.float64)).T @ np.abs(Y.astype(np.float64))
    for sym in (False, True):
        G = h.bdot(_dev(X), _dev(Y), sym=sym).cpu().numpy()
        if sym:
            iu = np.triu_indices(s)
            assert np.all(np.abs(G[iu] - ref[iu]) <= 2e-6 * bound[iu]), (n, s)
            assert np.array_equal(G, G.T)
        else:
            assert np.all(np.abs(G - ref) <= 2e-6 * bound), (n, s)


def test_bdot_fp32_widths_sharing_a_kernel_interleaved(h):
    # s = 12 and s = 16 run the same kernel with different shared memory:
    # a larger size after a smaller one must still launch
    g = np.random.default_rng(5)
    for s in (16, 12, 16, 12, 13, 16):
        X = g.integers(-4, 4, (5000, s)).astype(np.float32)
        for sym in (False, True):
            G = h.bdot(_dev(X), _dev(X), sym=sym).cpu().numpy()
            assert np.array_equal(G, X.astype(np.float64).T @ X.astype(np.float64)), (s, sym)


def test_bdot_fp32_integer_bit_exact(h):
    # small integers: every float product and partial sum is exact
    g = np.random.default_rng(8)
    for s in (4, 16, 32, 5):
        X = g.integers(-8, 8, (70001, s)).astype(np.float32)
        Y = g.integers(-8, 8, (70001, s)).astype(np.float32)
        G = h.bdot(_dev(X), _dev(Y)).cpu().numpy()
        assert np.array_equal(G, X.astype(np.float64).T @ Y.astype(np.float64)), s


@pytest.mark.parametrize("n,s", [(8, 8), (100, 3), (515, 8), (5157, 4), (5157, 32), (70001, 32),
                                 (300007, 8), (4096, 1)])
def test_tsqr_matches_householder(h, n, s):
    X = np.random.default_rng(n * 7 + s).standard_normal((n, s))
    Y, sig = h.tsqr(_dev(X))
    Y = Y.cpu().numpy(); sig = sig.cpu().numpy()
    Yr, Rr = oracle.householder_qr(X)
    assert np.allclose(np.tril(sig, -1), 0.0, atol=0) and np.all(np.diag(sig) >= 0)
    assert np.abs(sig - Rr).max() <= 1e-12 * np.abs(Rr).max()
    assert np.abs(Y - Yr).max() <= 1e-11
    assert np.abs(Y.T @ Y - np.eye(s)).max() <= 1e-13 * max(1, n / 1000)


def test_tsqr_in_place_and_rank_deficient(h):
    g = np.random.default_rng(11)
    X = g.standard_normal((3000, 6))
    X[:, 3] = X[:, 1]
    X[:, 5] = 0.0
    Xd = _dev(X)
    Y, sig = h.tsqr(Xd, Xd)          # Y aliases X
    Y = Y.cpu().numpy(); sig = sig.cpu().numpy()
    assert np.abs(Y.T @ Y - np.eye(6)).max() <= 1e-12
    assert np.abs(Y @ sig - X).max() <= 1e-12 * np.abs(X).max()
    assert np.all(np.diag(sig) >= 0) and np.allclose(np.tril(sig, -1), 0)
    assert abs(sig[5, 5]) <= 1e-13 and abs(sig[3, 3]) <= 1e-12


@pytest.mark.parametrize("n,s", [(20000, 8), (100, 3), (1000, 1), (5157, 4), (40000, 12),
                                 (300007, 16), (70001, 32)])
def test_tsqr_fp32(h, n, s):
    # FP32 leaves (quad-layout apply for s % 4 == 0), FP64 tree
    X = np.random.default_rng(5 + n + s).standard_normal((n, s)).astype(np.float32)
    Y, sig = h.tsqr(_dev(X))
    Y = Y.cpu().numpy().astype(np.float64); sig = sig.cpu().numpy()
    _, Rr = oracle.householder_qr(X.astype(np.float64))
    assert np.allclose(np.tril(sig, -1), 0.0, atol=0) and np.all(np.diag(sig) >= 0)
    assert np.abs(sig - Rr).max() <= 1e-4 * np.abs(Rr).max(), (n, s)
    assert np.abs(Y.T @ Y - np.eye(s)).max() <= 1e-4, (n, s)
    assert np.abs(Y @ sig - X).max() <= 1e-4 * np.abs(X).max(), (n, s)


def test_adjoint_scatter_and_edge_grad(h):
    nx, ny, s = 23, 19, 5
    g = np.random.default_rng(6)
    ax = np.exp(0.5 * g.standard_normal((ny, nx + 1))); ay = np.exp(0.5 * g.standard_normal((ny + 1, nx)))
    A = W.edge2d5(nx, ny, ax, ay)
    Lam = g.standard_normal((A.n, s)); X = g.standard_normal((A.n, s))
    from paper_2104_02494_gb300.api import operator_from_problem
    pr = W.Problem("e", A, None, dict(kind="edge5", nx=nx, ny=ny, nz=1, ax=ax, ay=ay))
    opc = operator_from_problem(h, pr, "csr")
    gs = h.adjoint_scatter(opc, _dev(Lam), _dev(X)).cpu().numpy()
    ref = oracle.adjoint_scatter(A, Lam, X)
    assert np.abs(gs - ref).max() <= 1e-13 * np.abs(ref).max()
    ops = operator_from_problem(h, pr, "stencil")
    ge = h.edge_theta_grad(ops, _dev(Lam), _dev(X)).cpu().numpy()
    gx, gy = oracle.edge_theta_grad(nx, ny, ax, ay, Lam, X)
    refe = np.concatenate([gx.ravel(), gy.ravel()])
    assert np.abs(ge - refe).max() <= 1e-13 * np.abs(refe).max()


def test_full_size_laplace_spmm_sampled_rows(h):
    """128^3 Laplacian, s = 8, stencil and CSR, in the bench's launch configuration."""
    from paper_2104_02494_gb300.api import operator_from_problem
    prob = W.problem("laplace3d", s=8)
    P = prob.B
    Pd = _dev(P)
    rows = np.random.default_rng(0).choice(prob.A.n, 2000, replace=False)
    rows = np.concatenate([rows, [0, prob.A.n - 1, 128 * 128 - 1, prob.A.n // 2]])
    A = prob.A
    for use in ("stencil", "csr"):
        op = operator_from_problem(h, prob, use)
        Q = h.spmm(op, Pd).cpu().numpy()
        for r in rows:
            cols = A.col[A.row_ptr[r]:A.row_ptr[r + 1]]
            vals = A.val[A.row_ptr[r]:A.row_ptr[r + 1]]
            ref = vals @ P[cols]
            bound = np.abs(vals) @ np.abs(P[cols])
            assert np.all(np.abs(Q[r] - ref) <= 1e-14 * bound), (use, r)
        op.close()
