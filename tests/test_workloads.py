"""Pins for the seeded problem generators (the operators A and blocks B)."""
import numpy as np
import pytest

import workloads as W


def test_nnz_formulas():
    # 5n - 4N (2D) and 7n - 6N^2 (3D) stored entries with Dirichlet boundaries
    for N in (3, 7, 16):
        assert W.lap2d5(N, N).nnz == 5 * N * N - 4 * N
        assert W.lap3d7(N, N, N).nnz == 7 * N ** 3 - 6 * N * N
    assert W.lap2d5(64, 64).nnz == 20224


def test_laplacian_closed_form_eigenvalues():
    nx, ny, nz = 4, 5, 3
    A = W.lap3d7(nx, ny, nz).to_dense()
    assert np.array_equal(A, A.T)
    lam = lambda N: 2 - 2 * np.cos(np.pi * np.arange(1, N + 1) / (N + 1))
    ev = (lam(nx)[None, None, :] + lam(ny)[None, :, None] + lam(nz)[:, None, None]).ravel()
    np.testing.assert_allclose(np.sort(ev), np.linalg.eigvalsh(A), rtol=0, atol=1e-12)


def _dense_from_stencil_loops(nx, ny, nz, coef):
    n = nx * ny * nz
    A = np.zeros((n, n))
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * (y + ny * z)
                for c, (dx, dy, dz) in zip(coef, offs):
                    X, Y, Z = x + dx, y + dy, z + dz
                    if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
                        A[i, X + nx * (Y + ny * Z)] = c
    return A


def test_const7_matches_loop_assembly():
    c = W.convdiff3d7_coeffs(5)
    A = W.const7(5, 4, 3, c)
    np.testing.assert_array_equal(A.to_dense(), _dense_from_stencil_loops(5, 4, 3, c))
    # CSR columns sorted inside each row
    for i in range(A.n):
        cols = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0)


def test_convdiff_upwind_signs():
    c = W.convdiff3d7_coeffs(96)
    h = 1 / 97
    assert c[0] == pytest.approx(6 + h * 10 * 1.75)
    assert c[1] == pytest.approx(-1 - h * 10) and c[2] == -1.0
    assert sum(c) == pytest.approx(0.0, abs=1e-14)   # row sum zero in the interior


def test_diff3d7_var_brute_force():
    nx, ny, nz = 3, 4, 2
    k = np.random.default_rng(5).uniform(0.5, 2.0, nx * ny * nz)
    A = W.diff3d7_var(nx, ny, nz, k).to_dense()
    n = nx * ny * nz
    ref = np.zeros((n, n))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * (y + ny * z)
                for dx, dy, dz in [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]:
                    X, Y, Z = x + dx, y + dy, z + dz
                    if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
                        j = X + nx * (Y + ny * Z)
                        f = 2 * k[i] * k[j] / (k[i] + k[j])
                        ref[i, j] -= f; ref[i, i] += f
                    else:
                        ref[i, i] += 2 * k[i]
    np.testing.assert_allclose(A, ref, rtol=1e-15, atol=0)
    assert np.all(np.linalg.eigvalsh(A) > 0)


def test_edge2d5_sum_of_edge_laplacians():
    nx, ny = 4, 3
    g = np.random.default_rng(0)
    ax = np.exp(g.standard_normal((ny, nx + 1))); ay = np.exp(g.standard_normal((ny + 1, nx)))
    A = W.edge2d5(nx, ny, ax, ay).to_dense()
    n = nx * ny
    ref = np.zeros((n, n))
    idx = lambda x, y: x + nx * y
    for y in range(ny):
        for x in range(nx + 1):
            a = ax[y, x]
            if 0 < x < nx:
                e = np.zeros(n); e[idx(x - 1, y)] = 1; e[idx(x, y)] = -1; ref += a * np.outer(e, e)
            else:
                i = idx(0 if x == 0 else nx - 1, y); ref[i, i] += a
    for y in range(ny + 1):
        for x in range(nx):
            a = ay[y, x]
            if 0 < y < ny:
                e = np.zeros(n); e[idx(x, y - 1)] = 1; e[idx(x, y)] = -1; ref += a * np.outer(e, e)
            else:
                i = idx(x, 0 if y == 0 else ny - 1); ref[i, i] += a
    np.testing.assert_allclose(A, ref, rtol=1e-14, atol=1e-14)


def test_rhs_prefix_property():
    B8 = W.normal_block(100, 8, 0, width=32)
    B32 = W.normal_block(100, 32, 0, width=32)
    np.testing.assert_array_equal(B8, B32[:, :8])
    assert B8.flags["C_CONTIGUOUS"]


def test_edge_problem_parameter_count():
    p = W.problem("edge2d", grid=16, s=2)
    assert p.stencil["ax"].size + p.stencil["ay"].size == 2 * 16 * 17
    assert p.A.nnz == 5 * 256 - 4 * 16
