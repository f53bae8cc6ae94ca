"""Seeded synthetic inputs for the block Krylov solvers.

This module is the only code shared by the CPU oracle (``oracle/``) and the GPU
path (``paper_2104_02494_gb300``).  It defines the *problems* — the sparse
operators A and the right-hand-side blocks B of the block system A X = B
(Dreier 2020, Ch. 3, Eq. "blocklinearsystem") — and nothing of the Krylov
methods themselves: no Gram matrices, no QR, no solver step lives here.

Layout conventions (shared by both sides):
  * grids are numbered lexicographically, x fastest:  i = x + nx*(y + ny*z);
  * block vectors are n x s row-major float64 arrays (the s right-hand sides
    of one grid point are contiguous, as in the thesis's SIMD block vector,
    Ch. 3.2);
  * CSR matrices use int32 row pointers / column indices with the column
    indices sorted ascending inside each row, float64 values.

Random numbers: ``numpy.random.default_rng(seed).standard_normal(shape)``
drawn row-major, so the first s columns of an n x 32 draw are the s-column
workload for every s <= 32.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "CSR", "Problem", "csr_from_triples", "lap2d5", "lap3d7", "const7",
    "convdiff3d7_coeffs", "diff3d7_var", "edge2d5", "normal_block",
    "problem", "CONFIGS",
]


@dataclass
class CSR:
    """Compressed sparse row matrix (int32 indices, float64 values)."""
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d


def csr_from_triples(n: int, rows, cols, vals) -> CSR:
    """Assemble a CSR matrix from (row, col, value) triples without duplicates."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate entries in triples")
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 range")
    return CSR(n, row_ptr.astype(np.int32), cols.astype(np.int32), vals)


# Offsets of the 7-point stencil in the order (center, -x, +x, -y, +y, -z, +z).
_OFFS7 = ((0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))


def _grid_index(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def const7(nx: int, ny: int, nz: int, coeffs) -> CSR:
    """Constant-coefficient 7-point stencil with homogeneous Dirichlet boundary.

    ``coeffs`` = (c_center, c_-x, c_+x, c_-y, c_+y, c_-z, c_+z); a neighbour
    outside the grid is dropped (its ghost value is zero).  With nz == 1 the
    z-couplings vanish and this is a 5-point 2D stencil.
    """
    c = np.asarray(coeffs, dtype=np.float64)
    assert c.shape == (7,)
    x, y, z = _grid_index(nx, ny, nz)
    idx = x + nx * (y + ny * z)
    rows, cols, vals = [], [], []
    for k, (dx, dy, dz) in enumerate(_OFFS7):
        xx, yy, zz = x + dx, y + dy, z + dz
        ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        rows.append(idx[ok])
        cols.append((xx + nx * (yy + ny * zz))[ok])
        vals.append(np.full(int(ok.sum()), c[k]))
    n = nx * ny * nz
    return csr_from_triples(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


LAPL7 = (6.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0)
LAPL5 = (4.0, -1.0, -1.0, -1.0, -1.0, 0.0, 0.0)


def lap2d5(nx: int, ny: int) -> CSR:
    """Unscaled 2D 5-point Poisson matrix (4 / -1), Dirichlet boundary."""
    return const7(nx, ny, 1, LAPL5)


def lap3d7(nx: int, ny: int, nz: int) -> CSR:
    """Unscaled 3D 7-point Laplacian (6 / -1), Dirichlet boundary."""
    return const7(nx, ny, nz, LAPL7)


def convdiff3d7_coeffs(N: int, pe: float = 10.0, direction=(1.0, 0.5, 0.25)):
    """Coefficients of -Lap(u) + v.grad(u) on the unit cube, first-order upwind.

    N^3 interior vertices, h = 1/(N+1), v = pe * direction (all components
    positive, so the upwind neighbour is the -d one).  The whole operator is
    multiplied by h^2 so that the entries are O(1):
      centre 6 + h (vx+vy+vz);  upwind (-d) -1 - h v_d;  downwind (+d) -1.
    """
    h = 1.0 / (N + 1)
    v = pe * np.asarray(direction, dtype=np.float64)
    return (6.0 + h * v.sum(), -1.0 - h * v[0], -1.0, -1.0 - h * v[1], -1.0,
            -1.0 - h * v[2], -1.0)


def diff3d7_var(nx: int, ny: int, nz: int, k: np.ndarray) -> CSR:
    """Cell-centred finite volumes for -div(k grad u), h = 1, Dirichlet u = 0.

    Interior face between cells i and j: harmonic average 2 k_i k_j / (k_i + k_j).
    Boundary face of cell i (ghost cell at distance h carrying u = 0): 2 k_i.
    Diagonal = sum of the cell's face coefficients, off-diagonal = -face.
    """
    k = np.asarray(k, dtype=np.float64).ravel()
    x, y, z = _grid_index(nx, ny, nz)
    idx = x + nx * (y + ny * z)
    n = nx * ny * nz
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for (dx, dy, dz) in _OFFS7[1:]:
        xx, yy, zz = x + dx, y + dy, z + dz
        ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        j = (xx + nx * (yy + ny * zz))
        face = np.where(ok, 2.0 * k * k[np.where(ok, j, 0)] / (k + k[np.where(ok, j, 0)]), 2.0 * k)
        diag += face
        rows.append(idx[ok]); cols.append(j[ok]); vals.append(-face[ok])
    rows.append(idx); cols.append(idx); vals.append(diag)
    return csr_from_triples(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def edge2d5(nx: int, ny: int, ax: np.ndarray, ay: np.ndarray) -> CSR:
    """2D 5-point diffusion with one coefficient per grid edge.

    ``ax`` has shape (ny, nx+1): ax[y, x] couples cell (x-1, y) and (x, y);
    the edges x = 0 and x = nx join a cell to its Dirichlet ghost.
    ``ay`` has shape (ny+1, nx): ay[y, x] couples (x, y-1) and (x, y).
    A = sum_e a_e (e_i - e_j)(e_i - e_j)^T + sum_{boundary e} a_e e_i e_i^T.
    """
    ax = np.asarray(ax, dtype=np.float64); ay = np.asarray(ay, dtype=np.float64)
    assert ax.shape == (ny, nx + 1) and ay.shape == (ny + 1, nx)
    n = nx * ny
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = x.ravel(); y = y.ravel(); idx = x + nx * y
    diag = ax[y, x] + ax[y, x + 1] + ay[y, x] + ay[y + 1, x]
    rows, cols, vals = [idx], [idx], [diag]
    m = x > 0
    rows.append(idx[m]); cols.append(idx[m] - 1); vals.append(-ax[y[m], x[m]])
    m = x < nx - 1
    rows.append(idx[m]); cols.append(idx[m] + 1); vals.append(-ax[y[m], x[m] + 1])
    m = y > 0
    rows.append(idx[m]); cols.append(idx[m] - nx); vals.append(-ay[y[m], x[m]])
    m = y < ny - 1
    rows.append(idx[m]); cols.append(idx[m] + nx); vals.append(-ay[y[m] + 1, x[m]])
    return csr_from_triples(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def normal_block(n: int, s: int, seed: int, width: Optional[int] = None) -> np.ndarray:
    """N(0,1) n x s block; the first s columns of a row-major n x width draw."""
    w = s if width is None else width
    return np.ascontiguousarray(np.random.default_rng(seed).standard_normal((n, w))[:, :s])


@dataclass
class Problem:
    """One synthetic workload: operator (CSR and stencil descriptor) plus RHS."""
    name: str
    A: CSR
    B: np.ndarray
    stencil: dict = field(default_factory=dict)   # kind + grid + coefficients
    extra: dict = field(default_factory=dict)


def _edge_fields(nx, ny, seed, sd=0.5):
    g = np.random.default_rng(seed)
    th_x = sd * g.standard_normal((ny, nx + 1))
    th_y = sd * g.standard_normal((ny + 1, nx))
    return th_x, th_y


def problem(name: str, s: int = None, grid: int = None, with_csr: bool = True) -> Problem:
    """Build one of the five workloads (optionally on a smaller grid).

    names: "poisson2d" (64^2, s=4), "laplace3d" (128^3, s in 1..32),
    "convdiff3d" (96^3, s=8), "vardiff3d" (192^3, s=16), "edge2d" (512^2, s=32).
    """
    if name == "poisson2d":
        N = grid or 64; s = s or 4
        A = lap2d5(N, N) if with_csr else None
        B = normal_block(N * N, s, 0)
        return Problem(name, A, B, dict(kind="const7", nx=N, ny=N, nz=1, coeffs=LAPL5))
    if name == "laplace3d":
        N = grid or 128; s = s or 8
        A = lap3d7(N, N, N) if with_csr else None
        B = normal_block(N ** 3, s, 0, width=max(32, s))
        return Problem(name, A, B, dict(kind="const7", nx=N, ny=N, nz=N, coeffs=LAPL7))
    if name == "convdiff3d":
        N = grid or 96; s = s or 8
        c = convdiff3d7_coeffs(N)
        A = const7(N, N, N, c) if with_csr else None
        B = normal_block(N ** 3, s, 0)
        return Problem(name, A, B, dict(kind="const7", nx=N, ny=N, nz=N, coeffs=c))
    if name == "vardiff3d":
        N = grid or 192; s = s or 16
        g = np.random.default_rng(1).standard_normal(N ** 3)
        k = np.exp(1.5 * g)
        A = diff3d7_var(N, N, N, k) if with_csr else None
        B = normal_block(N ** 3, s, 0)
        return Problem(name, A, B, dict(kind="var7", nx=N, ny=N, nz=N, k=k))
    if name == "edge2d":
        N = grid or 512; s = s or 32
        th_x, th_y = _edge_fields(N, N, 1)
        ax, ay = np.exp(th_x), np.exp(th_y)
        A = edge2d5(N, N, ax, ay) if with_csr else None
        B = normal_block(N * N, s, 0)
        Xt = normal_block(N * N, s, 2)
        return Problem(name, A, B, dict(kind="edge5", nx=N, ny=N, nz=1, ax=ax, ay=ay),
                       extra=dict(theta_x=th_x, theta_y=th_y, X_target=Xt))
    raise KeyError(name)


# Paper-shaped workload table: (name, grid, s values, solver, tolerance).
CONFIGS = {
    "poisson2d": dict(grid=64, s=(4,), solver="bcg", tol=1e-8, prec="fp64"),
    "laplace3d": dict(grid=128, s=(1, 4, 8, 16, 32), solver="bcg", tol=1e-8, prec="fp64"),
    "convdiff3d": dict(grid=96, s=(8,), solver="bbicgstab/bgmres30", tol=1e-8, prec="fp64"),
    "vardiff3d": dict(grid=192, s=(16,), solver="bcg-ir", tol=1e-10, prec="fp32+ir"),
    "edge2d": dict(grid=512, s=(32,), solver="bcg+adjoint", tol=1e-8, prec="fp64"),
}
