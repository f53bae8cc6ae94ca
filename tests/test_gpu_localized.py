"""GPU parity of BGMRes with the localized Arnoldi orthonormalisation (Ch. 9.3).

The GPU's row tiles are the FP64 TSQR leaf tiles (256 x 64 / next_pow2(s) rows,
256 x 32 / next_pow2(s) for s <= 4); the oracle runs the same tiling.  Checked:
the iterate after the first Arnoldi steps against the oracle's localized
BGMRes with the same tree fan-in (1e-11), converged solves against block MGS
(same step count, true residual at the tolerance), one tile (no tree) and tile
counts that leave nodes with fewer children, and the unsupported shapes.
"""
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


def _tile(s):
    sw = 1
    while sw < s:
        sw *= 2
    return 256 * (32 if sw <= 4 else 64) // sw


def _fanin(s, restart):
    """The library's tree fan-in: the widest of 8, 4, 2 whose node fits 200 KB of shared memory."""
    mx = restart + 1
    for F in (8, 4):
        cap = F * mx * s * s
        if 8 * (cap + max(cap, 256 * s) + s * s + 352) <= 200 * 1024:
            return F
    return 2


def _op(h, prob, use="stencil"):
    from paper_2104_02494_gb300.api import operator_from_problem
    return operator_from_problem(h, prob, use)


@pytest.mark.parametrize("grid,s", [(24, 8), (24, 4), (24, 16), (24, 3), (10, 8), (21, 1)])
def test_localized_first_steps_and_final(h, grid, s):
    prob = W.problem("convdiff3d", grid=grid, s=s)
    op = _op(h, prob)
    tile = _tile(s)
    for k in (1, 3, 8):
        X, info = h.solve("bgmres", op, _dev(prob.B), tol=0.0, maxit=k, restart=10, ortho="localized")
        ref = oracle.bgmres(prob.A, prob.B, tol=0.0, restart=10, maxit=k, ortho="localized", tile_rows=tile,
                            fanin=_fanin(s, 10))
        assert info.iters == k
        assert _rel(X.cpu().numpy(), ref.X) <= 1e-11, (k, _rel(X.cpu().numpy(), ref.X))
    X, info = h.solve("bgmres", op, _dev(prob.B), tol=1e-8, maxit=400, restart=10, ortho="localized")
    X2, info2 = h.solve("bgmres", op, _dev(prob.B), tol=1e-8, maxit=400, restart=10, ortho="mgs")
    assert info.converged and info2.converged and abs(info.iters - info2.iters) <= 1
    true = oracle.col_norms(prob.B - oracle.spmm(prob.A, X.cpu().numpy())) / oracle.col_norms(prob.B)
    assert true.max() <= 1.5e-8
    op.close()


@pytest.mark.parametrize("s,restart", [(2, 1), (8, 2), (8, 30)])
def test_localized_restart_lengths(h, s, restart):
    """Short and long cycles (restart 1: one basis vector per cycle)."""
    prob = W.problem("convdiff3d", grid=20, s=s)
    op = _op(h, prob)
    ref = oracle.bgmres(prob.A, prob.B, tol=0.0, restart=restart, maxit=6, ortho="localized",
                        tile_rows=_tile(s), fanin=_fanin(s, restart))
    X, info = h.solve("bgmres", op, _dev(prob.B), tol=0.0, maxit=6, restart=restart, ortho="localized")
    assert info.iters == 6 and _rel(X.cpu().numpy(), ref.X) <= 1e-11
    op.close()


def test_localized_unsupported_shapes(h):
    from paper_2104_02494_gb300.api import BkError
    prob = W.problem("convdiff3d", grid=24, s=32)
    op = _op(h, prob)
    with pytest.raises(BkError):                       # s > 16
        h.solve("bgmres", op, _dev(prob.B), tol=1e-8, maxit=10, restart=10, ortho="localized")
    op.close()
    n = 2 * 2048 + 3                                   # last tile of 3 rows < s = 8
    A = W.csr_from_triples(n, np.arange(n), np.arange(n), np.full(n, 2.0))
    dv = lambda a: torch.from_numpy(np.asarray(a)).cuda()
    op = h.op_csr(dv(A.row_ptr), dv(A.col), dv(A.val))
    B = W.normal_block(n, 8, 0)
    with pytest.raises(BkError):
        h.solve("bgmres", op, _dev(B), tol=1e-8, maxit=10, restart=10, ortho="localized")
    op.close()
