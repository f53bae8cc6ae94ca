"""The grid-wide reduction of the Gram kernels on both of its levels.

A Gram kernel's CTAs store their partial sums; the last CTA sums them (one level), or, with
many partial values, the last CTA of each group of 16 CTAs sums its group and the last group
sums the group sums (two levels).  Integer-valued blocks make every product and partial sum
exact, so any order gives the same Gram and a lost, doubled or misplaced partial shows as a
wrong entry.  The widths and row counts below put the grids on either side of the switch:
FP32 s = 32 streams 192 rows per CTA step, s = 16 384 rows, so n = 192 * 17 gives a grid of
17 CTAs (groups of 16 and 1), n = 192 * 33 + 5 a grid of 34 (16, 16, 2).
"""
import numpy as np
import pytest
import torch

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


CASES = [
    (np.float32, 32, 192 * 17 - 7),
    (np.float32, 32, 192 * 33 + 5),
    (np.float32, 32, 192 * 160),
    (np.float32, 16, 384 * 17),
    (np.float32, 16, 384 * 300 + 1),
    (np.float32, 8, 300007),
    (np.float64, 8, 300007),
    (np.float64, 16, 200003),
    (np.float64, 32, 100003),
    (np.float64, 5, 1000003),
]


@pytest.mark.parametrize("dtype,s,n", CASES)
def test_gram_integer_exact_on_both_levels(h, dtype, s, n):
    g = np.random.default_rng(n + s)
    X = g.integers(-8, 8, (n, s)).astype(dtype)
    Y = g.integers(-8, 8, (n, s)).astype(dtype)
    ref = X.astype(np.float64).T @ Y.astype(np.float64)
    G = h.bdot(_dev(X), _dev(Y)).cpu().numpy()
    assert np.array_equal(G, ref), (dtype, s, n)
    ref_xx = X.astype(np.float64).T @ X.astype(np.float64)
    G = h.bdot(_dev(X), _dev(X), sym=True).cpu().numpy()
    assert np.array_equal(G, ref_xx), (dtype, s, n)


@pytest.mark.parametrize("dtype,s,n", [(np.float32, 32, 192 * 160), (np.float64, 16, 200003)])
def test_gram_two_levels_reproducible(h, dtype, s, n):
    g = np.random.default_rng(7)
    X = _dev(g.standard_normal((n, s)).astype(dtype))
    Y = _dev(g.standard_normal((n, s)).astype(dtype))
    a = h.bdot(X, Y).cpu().numpy()
    for _ in range(3):
        assert np.array_equal(h.bdot(X, Y).cpu().numpy(), a)
    b = h.bdot(X, X, sym=True).cpu().numpy()
    assert np.array_equal(h.bdot(X, X, sym=True).cpu().numpy(), b)
    assert np.array_equal(b, b.T)


def test_fused_operator_gram_integer_exact_at_32_columns(h):
    # the marching kernel's tensor-core Gram at s = 32 reduces 528 values per CTA
    import oracle
    import workloads as W
    from paper_2104_02494_gb300.api import operator_from_problem
    prob = W.problem("laplace3d", s=32, grid=40, with_csr=True)
    op = operator_from_problem(h, prob, "stencil")
    g = np.random.default_rng(11)
    P = g.integers(-4, 4, (prob.B.shape[0], 32)).astype(np.float32)
    Pd = _dev(P)
    Q = torch.empty_like(Pd)
    G = torch.empty(32, 32, dtype=torch.float64, device="cuda")
    h.spmm_gram(op, Pd, Q, G=G)
    Qref = oracle.spmm(prob.A, P.astype(np.float64))
    assert np.array_equal(Q.cpu().numpy().astype(np.float64), Qref)
    assert np.array_equal(G.cpu().numpy(), P.astype(np.float64).T @ Qref)
    op.close()
