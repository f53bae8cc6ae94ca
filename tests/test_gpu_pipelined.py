"""Pipelined FP32 kernels (asynchronous bulk copies into a shared-memory ring).

The marching stencil kernel (operator product Q = A P, alone and with the Gram
P^T Q fused, the alpha pass of Alg. "bcgaro") and the streaming block inner
product, on grids that split into many tiles and z-segments (so that both
marching directions and ragged edge tiles occur), on 2D grids, for every quad
width s = 4, 8, ..., 32 (non-powers of two leave lanes idle) and at full size.
References come from the oracle on the same inputs:
  * integer-valued inputs (small integers): bit-exact, products and partial
    sums are exact in FP32, the TF32 split and FP64;
  * random inputs: 2e-6 of the magnitude bound |A||P| (Q) and |P|^T|A||P| (G).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

# (nx, ny, nz); nz = 1 is a 2D grid (marched along y)
GRIDS = [(40, 33, 29), (130, 3, 7), (1, 1, 50), (257, 2, 3), (17, 23, 1), (3, 300, 1)]
WIDTHS = [4, 8, 12, 16, 20, 32]


@pytest.fixture(scope="module")
def h():
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle
    build()
    with Handle(0) as hh:
        yield hh


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _lap_op(h, nx, ny, nz):
    from paper_2104_02494_gb300.api import operator_from_problem
    prob = W.Problem("lap", W.const7(nx, ny, nz, W.LAPL7), None,
                     dict(kind="const7", nx=nx, ny=ny, nz=nz, coeffs=W.LAPL7))
    return prob.A, operator_from_problem(h, prob, "stencil")


def _var7_op(h, nx, ny, nz, seed=1):
    from paper_2104_02494_gb300.api import operator_from_problem
    k = np.exp(1.5 * np.random.default_rng(seed).standard_normal(nx * ny * nz))
    prob = W.Problem("vd", W.diff3d7_var(nx, ny, nz, k), None, dict(kind="var7", nx=nx, ny=ny, nz=nz, k=k))
    return prob.A, operator_from_problem(h, prob, "stencil")


def _edge5_op(h, nx, ny, seed=2):
    from paper_2104_02494_gb300.api import operator_from_problem
    g = np.random.default_rng(seed)
    ax = np.exp(0.5 * g.standard_normal((ny, nx + 1))); ay = np.exp(0.5 * g.standard_normal((ny + 1, nx)))
    prob = W.Problem("ed", W.edge2d5(nx, ny, ax, ay), None, dict(kind="edge5", nx=nx, ny=ny, nz=1, ax=ax, ay=ay))
    return prob.A, operator_from_problem(h, prob, "stencil")


def _absbound(A, P):
    Aabs = W.CSR(A.n, A.row_ptr, A.col, np.abs(A.val))
    return oracle.spmm(Aabs, np.abs(P))


@pytest.mark.parametrize("grid", GRIDS)
def test_march_laplacian_integer_bit_exact(h, grid):
    A, op = _lap_op(h, *grid)
    for s in WIDTHS:
        P = np.random.default_rng(s).integers(-8, 8, (A.n, s)).astype(np.float32)
        Pd = _dev(P)
        ref = oracle.spmm(A, P.astype(np.float64))
        Q = h.spmm(op, Pd).cpu().numpy().astype(np.float64)
        assert np.array_equal(Q, ref), (grid, s)
        Q2, G = h.spmm_gram(op, Pd, sym=True)
        assert np.array_equal(Q2.cpu().numpy().astype(np.float64), ref), (grid, s)
        Gref = P.astype(np.float64).T @ ref
        assert np.array_equal(G.cpu().numpy(), Gref), (grid, s)
    op.close()


@pytest.mark.parametrize("grid", [(40, 33, 29), (257, 2, 3), (5, 70, 11)])
def test_march_var7_fp32(h, grid):
    A, op = _var7_op(h, *grid)
    for s in WIDTHS:
        P = np.random.default_rng(10 + s).standard_normal((A.n, s)).astype(np.float32)
        P64 = P.astype(np.float64)
        ref = oracle.spmm(A, P64)
        bound = _absbound(A, P64)
        Q, G = h.spmm_gram(op, _dev(P), sym=True)
        Q = Q.cpu().numpy().astype(np.float64)
        assert (np.abs(Q - ref) <= 2e-6 * bound + 1e-30).all(), (grid, s)
        Gref = P64.T @ ref
        Gbound = np.abs(P64).T @ bound
        iu = np.triu_indices(s)
        Gg = G.cpu().numpy()
        assert (np.abs(Gg[iu] - Gref[iu]) <= 2e-6 * Gbound[iu]).all(), (grid, s)
        assert np.array_equal(Gg, Gg.T)
    op.close()


@pytest.mark.parametrize("grid", [(70, 45), (300, 3), (1, 90)])
def test_march_edge5_fp32(h, grid):
    A, op = _edge5_op(h, *grid)
    for s in WIDTHS:
        P = np.random.default_rng(20 + s).standard_normal((A.n, s)).astype(np.float32)
        P64 = P.astype(np.float64)
        ref = oracle.spmm(A, P64)
        bound = _absbound(A, P64)
        Q = h.spmm(op, _dev(P)).cpu().numpy().astype(np.float64)
        assert (np.abs(Q - ref) <= 2e-6 * bound + 1e-30).all(), (grid, s)
        Q2, G = h.spmm_gram(op, _dev(P), sym=True)
        Gref = P64.T @ ref
        Gbound = np.abs(P64).T @ bound
        iu = np.triu_indices(s)
        assert (np.abs(G.cpu().numpy()[iu] - Gref[iu]) <= 2e-6 * Gbound[iu]).all(), (grid, s)
    op.close()


def test_march_convdiff_fp32_and_repeat(h):
    # asymmetric constant stencil (upwind): the -z / +z coefficients differ, so a
    # segment marching downwards must still pair each plane with the right one
    from paper_2104_02494_gb300.api import operator_from_problem
    nx, ny, nz = 36, 31, 40
    c = W.convdiff3d7_coeffs(nx)
    prob = W.Problem("cd", W.const7(nx, ny, nz, c), None, dict(kind="const7", nx=nx, ny=ny, nz=nz, coeffs=c))
    op = operator_from_problem(h, prob, "stencil")
    for s in (8, 16, 32):
        P = np.random.default_rng(s).standard_normal((prob.A.n, s)).astype(np.float32)
        ref = oracle.spmm(prob.A, P.astype(np.float64))
        bound = _absbound(prob.A, P.astype(np.float64))
        Pd = _dev(P)
        Q1, G1 = h.spmm_gram(op, Pd)
        Q2, G2 = h.spmm_gram(op, Pd)
        assert torch.equal(Q1, Q2) and torch.equal(G1, G2)     # fixed reduction order
        assert (np.abs(Q1.cpu().numpy() - ref) <= 2e-6 * bound + 1e-30).all(), s
    op.close()


@pytest.mark.parametrize("s", [8, 16, 32])
def test_march_full_size_laplace128(h, s):
    # the benchmark's grid: integer block, Q and G exact
    A, op = _lap_op(h, 128, 128, 128)
    P = np.random.default_rng(s).integers(-8, 8, (A.n, s)).astype(np.float32)
    ref = oracle.spmm(A, P.astype(np.float64))
    Q, G = h.spmm_gram(op, _dev(P), sym=True)
    assert np.array_equal(Q.cpu().numpy().astype(np.float64), ref), s
    assert np.array_equal(G.cpu().numpy(), P.astype(np.float64).T @ ref), s
    op.close()


def test_stream_bdot_full_size_and_ragged(h):
    # chunked 1D bulk copies: n not a multiple of the chunk, several chunks per CTA
    g = np.random.default_rng(9)
    for n, s in ((2_097_152 + 37, 16), (1_000_003, 32), (333_333, 4), (77, 8)):
        X = g.integers(-8, 8, (n, s)).astype(np.float32)
        Y = g.integers(-8, 8, (n, s)).astype(np.float32)
        Xd, Yd = _dev(X), _dev(Y)
        X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
        assert np.array_equal(h.bdot(Xd, Yd).cpu().numpy(), X64.T @ Y64), (n, s)
        G = h.bdot(Xd, Xd, sym=True).cpu().numpy()
        assert np.array_equal(G, X64.T @ X64), (n, s)
