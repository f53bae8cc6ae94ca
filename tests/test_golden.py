"""The stored expected values of tests/golden/.

bcg_poisson2d_12x11_s3.json is written by tests/golden/make_golden.py from the oracle alone:
the oracle still reproduces it (CPU), and the GPU solvers match it (-m gpu).
gmres_cyclic_shift.json is the thesis's own worked example (Ch. 2, Ex. "nonconverging_gmres"):
GMRes on the cyclic shift with b = e_1 cannot improve on x = 0 before n steps and is exact at n.

Residual histories are compared relatively (1e-9 on the CPU, where only the BLAS build may
differ; 1e-8 on the GPU, whose Gram summation order differs and whose FP64 BCG normalises
by CholeskyQR2), decisions and iteration counts exactly.  Each entry may also be off by
1e-15 absolutely: the history is max_i ||R-bar sigma e_i|| / ||R0_i||, and the normaliser's
rounding in sigma is relative to ||sigma|| (about 1 in these units), not to a converged
column's own small norm (near 1e-11 at the end; another BLAS build on an Arm host moved
the preconditioned case's tail by 3e-8 relative).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "bcg_poisson2d_12x11_s3.json")))


def _problems():
    A = W.lap2d5(12, 11)
    B = W.normal_block(A.n, 3, 0)
    k = np.exp(1.5 * np.random.default_rng(5).standard_normal(125))
    Av = W.diff3d7_var(5, 5, 5, k)
    Bv = W.normal_block(Av.n, 3, 1)
    return A, B, Av, Bv


CASES = [("bcg_eta_inf", "bcg", math.inf, False, False), ("bcg_eta_0", "bcg", 0.0, False, False),
         ("bcg_eta_1e4", "bcg", 1e4, False, False), ("bcg_1r_eta_inf", "bcg_1r", math.inf, False, False),
         ("bcg_jacobi_vardiff_eta_inf", "bcg", math.inf, True, True)]


def _check(got_hist, got_dec, got_iters, ref, tol, floor=0.0):
    assert got_iters == ref["iters"]
    assert list(got_dec) == ref["decisions"]
    h = np.array(got_hist[:len(ref["history"])])
    r = np.array(ref["history"])
    assert np.all(np.abs(h - r) <= tol * np.abs(r) + floor), np.abs(h / r - 1).max()


@pytest.mark.parametrize("key,fn,eta,jacobi,var", CASES)
def test_oracle_reproduces_golden(key, fn, eta, jacobi, var):
    A, B, Av, Bv = _problems()
    M, R = (Av, Bv) if var else (A, B)
    w = oracle.jacobi_inverse_diagonal(M) if jacobi else None
    r = getattr(oracle, fn)(M, R, tol=1e-10, maxit=500, eta=eta, Minv=w)
    _check(r.history, r.decisions, r.iters, GOLD[key], 1e-9, floor=1e-15)


@pytest.mark.gpu
@pytest.mark.parametrize("key,fn,eta,jacobi,var", CASES)
def test_gpu_matches_golden(key, fn, eta, jacobi, var):
    import torch
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle
    build()
    A, B, Av, Bv = _problems()
    M, R = (Av, Bv) if var else (A, B)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with Handle(0) as h:
        op = h.op_csr(dv(M.row_ptr), dv(M.col), dv(M.val))
        P = h.op_jacobi(op) if jacobi else None
        X, info = h.solve("bcg", op, dv(R), tol=1e-10, maxit=500, eta=eta, precond=P,
                          one_reduction=(fn == "bcg_1r"))
        _check(info.history, info.decisions, info.iters, GOLD[key], 1e-8, floor=1e-15)
        ref_row = np.array(GOLD[key]["X_first_row"])
        assert np.abs(X.cpu().numpy()[0] - ref_row).max() <= 1e-9 * np.abs(ref_row).max()
        if P is not None:
            P.close()
        op.close()


CYCLIC = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "gmres_cyclic_shift.json")))


def _cyclic(n, transposed):
    """The example's matrix: the printed form (superdiagonal and bottom-left corner) or its
    transpose (subdiagonal and top-right corner, the form the example's text describes)."""
    rows = list(range(n - 1)) + [n - 1]
    cols = list(range(1, n)) + [0]
    if transposed:
        rows, cols = cols, rows
    return W.csr_from_triples(n, rows, cols, np.ones(n))


@pytest.mark.parametrize("n", CYCLIC["n"])
@pytest.mark.parametrize("transposed", [False, True])
@pytest.mark.parametrize("ortho", ["mgs", "cgs2", "localized"])
def test_oracle_gmres_stalls_on_the_cyclic_shift(n, transposed, ortho):
    A = _cyclic(n, transposed)
    b = np.zeros((n, 1)); b[0, 0] = 1.0
    for k in range(1, n):
        r = oracle.bgmres(A, b, tol=0.0, restart=n, maxit=k, ortho=ortho, tile_rows=n)
        assert np.abs(r.X).max() <= 1e-14, (k, np.abs(r.X).max())
        assert abs(r.history[-1] - CYCLIC["relative_residual_before_n"]) <= 1e-14
    r = oracle.bgmres(A, b, tol=0.0, restart=n, maxit=n, ortho=ortho, tile_rows=n)
    sol = np.zeros(n); sol[n - 1 if transposed else 1] = 1.0        # e_n resp. e_2
    assert np.abs(r.X[:, 0] - sol).max() <= 1e-13
    assert r.history[-1] <= 1e-13


@pytest.mark.parametrize("n", CYCLIC["n"])
def test_oracle_bbicgstab_breaks_down_on_the_cyclic_shift(n):
    """BiCGStab's first coefficient divides by r0^T A r0 = A[0][0] = 0: a breakdown, X untouched."""
    A = _cyclic(n, False)
    b = np.zeros((n, 1)); b[0, 0] = 1.0
    for eta in (0.0, math.inf):
        r = oracle.bbicgstab(A, b, tol=1e-12, maxit=2 * n, eta=eta)
        assert r.status == "breakdown" and r.iters == 0 and np.all(r.X == 0.0)
