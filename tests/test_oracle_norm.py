"""Pins of the oracle's stopping measures (reading c2).

The thesis stops on "||R|| < tol" (Ch. 4.1) without naming the norm.  The
default measure is the reduction in every column, max_i ||R_i|| / ||R^0_i||;
the Frobenius measure ||R||_F / ||R^0||_F is selectable (norm="fro").  Pinned
here by closed forms, by s = 1 (both measures are the same number), by the
first iteration at which the explicitly recomputed residual B - A X^k crosses
tol in the Frobenius norm, and by the ordering ||R||_F / ||R^0||_F <=
max_i ||R_i|| / ||R^0_i|| (so a Frobenius run never stops later).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle.blockops import spmm, stop_measure


def test_stop_measure_closed_forms():
    relres = np.array([0.5, 0.1, 0.0])
    n0 = np.array([2.0, 1.0, 0.0])
    assert stop_measure(relres, n0, "max") == 0.5
    # ||R||_F^2 = (0.5 * 2)^2 + (0.1 * 1)^2 = 1.01, ||R^0||_F^2 = 5
    assert abs(stop_measure(relres, n0, "fro") - math.sqrt(1.01 / 5.0)) < 1e-15
    # equal relative residuals in every column: both measures agree
    assert abs(stop_measure([0.3, 0.3, 0.3], [1.0, 7.0, 2.0], "fro") - 0.3) < 1e-15
    assert stop_measure([0.0, 0.0], [0.0, 0.0], "fro") == 0.0
    with pytest.raises(ValueError):
        stop_measure(relres, n0, "l1")


def _poisson(N=20, s=4):
    p = W.problem("poisson2d", s=s, grid=N)
    return p.A, p.B


def _true_fro(A, B, X):
    return np.linalg.norm(B - spmm(A, X)) / np.linalg.norm(B)


def test_s1_both_measures_identical():
    A, B = _poisson(16, 1)
    for solve in (lambda nm: oracle.bcg(A, B, tol=1e-9, norm=nm),
                  lambda nm: oracle.bcg_1r(A, B, tol=1e-9, norm=nm),
                  lambda nm: oracle.bbicgstab(A, B, tol=1e-9, norm=nm),
                  lambda nm: oracle.bgmres(A, B, tol=1e-9, restart=20, norm=nm)):
        a, b = solve("max"), solve("fro")
        assert a.iters == b.iters and np.array_equal(a.X, b.X) and a.history == b.history


def test_bcg_fro_stops_at_first_true_crossing():
    A, B = _poisson(20, 4)
    tol = 1e-6
    K = 200
    free = oracle.bcg(A, B, tol=0.0, maxit=K, record_iterates=K)
    true = [_true_fro(A, B, Xk) for Xk in free.iterates]
    k_star = next(k for k, v in enumerate(true) if v <= tol) + 1
    assert true[k_star - 1] < tol * (1 - 1e-6) and true[k_star - 2] > tol * (1 + 1e-6)   # not borderline
    fro = oracle.bcg(A, B, tol=tol, norm="fro")
    mx = oracle.bcg(A, B, tol=tol, norm="max")
    assert fro.converged and fro.iters == k_star
    assert fro.iters <= mx.iters
    assert abs(fro.history[-1] - true[k_star - 1]) <= 1e-9 * tol + 1e-12 * true[k_star - 1] * 1e3


def test_bbicgstab_and_bgmres_fro():
    p = W.problem("convdiff3d", s=3, grid=8)
    tol = 1e-7
    for solve in (lambda nm: oracle.bbicgstab(p.A, p.B, tol=tol, eta=100.0, norm=nm),
                  lambda nm: oracle.bgmres(p.A, p.B, tol=tol, restart=15, norm=nm, ortho="cgs2")):
        fro, mx = solve("fro"), solve("max")
        assert fro.converged and mx.converged
        assert fro.iters <= mx.iters
        assert _true_fro(p.A, p.B, fro.X) <= tol * 1.01
        # the Frobenius run stopped at the first iteration whose tracked measure is below tol
        assert fro.history[-1] <= tol and all(h > tol for h in fro.history[:-1])


def test_ir_fro_outer_test():
    p = W.problem("vardiff3d", s=3, grid=8)
    fro = oracle.bcg_ir(p.A, p.B, tol=1e-10, norm="fro")
    mx = oracle.bcg_ir(p.A, p.B, tol=1e-10, norm="max")
    assert fro.converged and mx.converged and fro.outer <= mx.outer
    assert _true_fro(p.A, p.B, fro.X) <= 1e-10
