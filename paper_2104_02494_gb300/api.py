"""Python wrappers over the bkrylov C ABI (argument marshalling only).

Device blocks are torch CUDA tensors (n x s, row-major = contiguous);
host blocks may be numpy arrays or CPU tensors for the solvers, which then
copy them inside the C call.  Every computation runs in the library's CUDA
kernels.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L

_STENCIL = {"const7": L.BK_STENCIL_CONST7, "var7": L.BK_STENCIL_VAR7, "edge5": L.BK_STENCIL_EDGE5,
            "edge5_log": L.BK_STENCIL_EDGE5_LOG}
_PREC = {"fp64": L.BK_FP64, "fp32": L.BK_FP32, "fp32_ir": L.BK_FP32_IR}


class BkError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {L.status_string(status)} (status {status})")
        self.status = status


def _check(st: int, where: str):
    if st != L.BK_OK:
        raise BkError(st, where)


def _ptr(t) -> int:
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("blocks must be contiguous (row-major n x s)")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("blocks must be C-contiguous")
        return t.ctypes.data
    raise TypeError(type(t))


def _prec_of(t) -> int:
    dt = t.dtype
    if dt in (torch.float64, np.float64):
        return L.BK_FP64
    if dt in (torch.float32, np.float32):
        return L.BK_FP32
    raise TypeError(f"unsupported dtype {dt}")


class Handle:
    """bkrylov_create / bkrylov_destroy; bound to torch's current CUDA stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.lib = L.load()
        self.device = device
        st = stream if stream is not None else torch.cuda.current_stream(device)
        h = C.c_void_p()
        _check(self.lib.bkrylov_create(C.byref(h), device, C.c_void_p(st.cuda_stream or None)),
               "bkrylov_create")
        self.h = h
        self._ops = []

    def close(self):
        if self.h:
            for op in list(self._ops):
                op.close()
            self.lib.bkrylov_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- operators ----
    def op_csr(self, row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor) -> "Operator":
        n = row_ptr.numel() - 1
        if row_ptr.dtype != torch.int32 or col.dtype != torch.int32:
            raise TypeError("CSR row_ptr and col must be int32")
        A = C.c_void_p()
        _check(self.lib.bkrylov_op_csr(self.h, n, col.numel(), _ptr(row_ptr), _ptr(col), _ptr(val),
                                       _prec_of(val), C.byref(A)), "bkrylov_op_csr")
        op = Operator(self, A, n, keep=(row_ptr, col, val))
        self._ops.append(op)
        return op

    def op_stencil(self, kind: str, nx: int, ny: int, nz: int, coeffs) -> "Operator":
        A = C.c_void_p()
        k = _STENCIL[kind]
        if k == L.BK_STENCIL_CONST7:
            arr = (C.c_double * 7)(*[float(c) for c in coeffs])
            p = C.cast(arr, C.c_void_p)
            keep = (arr,)
        else:
            assert isinstance(coeffs, torch.Tensor) and coeffs.is_cuda and coeffs.dtype == torch.float64
            p = C.c_void_p(_ptr(coeffs))
            keep = (coeffs,)
        _check(self.lib.bkrylov_op_stencil(self.h, k, nx, ny, nz, p, C.byref(A)), "bkrylov_op_stencil")
        op = Operator(self, A, nx * ny * nz, keep=keep, kind=kind, grid=(nx, ny, nz))
        self._ops.append(op)
        return op

    def op_transpose(self, A: "Operator") -> "Operator":
        """A^T as an operator of its own (bkrylov_op_transpose: CSR and CONST7)."""
        At = C.c_void_p()
        _check(self.lib.bkrylov_op_transpose(self.h, A.ptr, C.byref(At)), "bkrylov_op_transpose")
        op = Operator(self, At, A.n, kind=A.kind, grid=A.grid)
        self._ops.append(op)
        return op

    def op_diag(self, d: torch.Tensor) -> "Operator":
        """Diagonal operator diag(d) (d: float64 CUDA vector, copied)."""
        assert d.is_cuda and d.dtype == torch.float64 and d.dim() == 1
        M = C.c_void_p()
        _check(self.lib.bkrylov_op_diag(self.h, d.numel(), _ptr(d), C.byref(M)), "bkrylov_op_diag")
        op = Operator(self, M, d.numel(), kind="diag")
        self._ops.append(op)
        return op

    def op_jacobi(self, A: "Operator") -> "Operator":
        """Point Jacobi preconditioner M^{-1} = diag(A)^{-1} as a diagonal operator."""
        M = C.c_void_p()
        _check(self.lib.bkrylov_op_jacobi(self.h, A.ptr, C.byref(M)), "bkrylov_op_jacobi")
        op = Operator(self, M, A.n, kind="diag")
        self._ops.append(op)
        return op

    # ---- single kernels ----
    def spmm(self, A: "Operator", P: torch.Tensor, Q: torch.Tensor | None = None) -> torch.Tensor:
        Q = torch.empty_like(P) if Q is None else Q
        _check(self.lib.bkrylov_spmm(self.h, A.ptr, P.shape[1], _ptr(P), _ptr(Q), _prec_of(P)),
               "bkrylov_spmm")
        return Q

    def spmm_gram(self, A: "Operator", P: torch.Tensor, Q: torch.Tensor | None = None, sym: bool = True,
                  G: torch.Tensor | None = None):
        """Q = A P and G = P^T Q in one pass (bkrylov_spmm_gram); returns (Q, G)."""
        s = P.shape[1]
        Q = torch.empty_like(P) if Q is None else Q
        G = torch.empty((s, s), dtype=torch.float64, device=P.device) if G is None else G
        _check(self.lib.bkrylov_spmm_gram(self.h, A.ptr, s, _ptr(P), _ptr(Q), _ptr(G), int(sym), _prec_of(P)),
               "bkrylov_spmm_gram")
        return Q, G

    def residual(self, A: "Operator", B: torch.Tensor, X: torch.Tensor,
                 R: torch.Tensor | None = None) -> torch.Tensor:
        R = torch.empty_like(B) if R is None else R
        _check(self.lib.bkrylov_residual(self.h, A.ptr, B.shape[1], _ptr(B), _ptr(X), _ptr(R),
                                         _prec_of(B)), "bkrylov_residual")
        return R

    def bdot(self, X: torch.Tensor, Y: torch.Tensor, sym: bool = False,
             G: torch.Tensor | None = None) -> torch.Tensor:
        n, s = X.shape
        G = torch.empty((s, s), dtype=torch.float64, device=X.device) if G is None else G
        _check(self.lib.bkrylov_bdot(self.h, n, s, _ptr(X), _ptr(Y), _ptr(G), int(sym), _prec_of(X)),
               "bkrylov_bdot")
        return G

    def tsqr(self, X: torch.Tensor, Y: torch.Tensor | None = None):
        n, s = X.shape
        Y = torch.empty_like(X) if Y is None else Y
        sig = torch.empty((s, s), dtype=torch.float64, device=X.device)
        _check(self.lib.bkrylov_tsqr(self.h, n, s, _ptr(X), _ptr(Y), _ptr(sig), _prec_of(X)),
               "bkrylov_tsqr")
        return Y, sig

    def adjoint_scatter(self, A: "Operator", Lam: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
        g = torch.empty(A.nnz, dtype=torch.float64, device=Lam.device)
        _check(self.lib.bkrylov_adjoint_scatter(self.h, A.ptr, Lam.shape[1], _ptr(Lam), _ptr(X), _ptr(g)),
               "bkrylov_adjoint_scatter")
        return g

    def edge_theta_grad(self, A: "Operator", Lam: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
        nx, ny, _ = A.grid
        g = torch.empty(ny * (nx + 1) + (ny + 1) * nx, dtype=torch.float64, device=Lam.device)
        _check(self.lib.bkrylov_edge_theta_grad(self.h, A.ptr, Lam.shape[1], _ptr(Lam), _ptr(X), _ptr(g)),
               "bkrylov_edge_theta_grad")
        return g

    def kappa_d(self, A: torch.Tensor) -> float:
        """kappa_D of an s x s symmetric float64 CUDA matrix (the adaptive criterion's)."""
        out = torch.empty(1, dtype=torch.float64, device=A.device)
        A = A.contiguous()
        _check(self.lib.bkrylov_kappa_d(self.h, A.shape[0], _ptr(A), _ptr(out)), "bkrylov_kappa_d")
        return float(out.item())

    def reortho_decision(self, A: torch.Tensor, eta: float, eps: float = 2.0 ** -52) -> bool:
        """The solvers' re-orthonormalisation decision for the s x s matrix A (float64, CUDA)."""
        out = torch.zeros(1, dtype=torch.int32, device=A.device)
        A = A.contiguous()
        _check(self.lib.bkrylov_reortho_decision(self.h, A.shape[0], _ptr(A), float(eta), float(eps), _ptr(out)),
               "bkrylov_reortho_decision")
        return bool(out.item())

    # ---- measurement ----
    def profile(self):
        """[(phase, total_ms, launches)] accumulated by solves run with profile=True."""
        out = []
        for i in range(self.lib.bkrylov_profile_count()):
            name, ms, nl = C.c_char_p(), C.c_double(), C.c_longlong()
            _check(self.lib.bkrylov_profile_get(self.h, i, C.byref(name), C.byref(ms), C.byref(nl)),
                   "bkrylov_profile_get")
            out.append((name.value.decode(), ms.value, nl.value))
        return out

    def profile_reset(self):
        _check(self.lib.bkrylov_profile_reset(self.h), "bkrylov_profile_reset")

    # ---- solvers ----
    def solve(self, method: str, A: "Operator", B, X=None, *, tol=1e-8, maxit=1000, eta=math.inf,
              prec="fp64", restart=30, ortho="mgs", ir_inner_tol=1e-5, ir_max_outer=30,
              forced_reortho=None, sync_every=0, record=True, profile=False, p=None, precond=None,
              one_reduction=False, norm="max", qr="cholqr2", replace_every=0):
        """Run bkrylov_solve_{bcg,bbicgstab,bgmres}; returns (X, SolveInfo).

        B, X: n x s blocks, float64 (prec "fp64", "fp32_ir") or float32 (prec "fp32"),
        on the device (torch CUDA tensors) or on the host (numpy / CPU tensors; copied
        inside the call).  X is updated in place and starts from zero when not given.
        ``p``: block size of the block-parallel subalgebra (BCG); ``precond``: an Operator
        applying M^{-1} (BCG, e.g. ``op_jacobi(A)``); ``one_reduction``: the 1R-BCG
        schedule; ``norm``: the stopping measure, "max" (every column) or "fro"; ``qr``:
        the normaliser of FP64 BCG, "cholqr2" (CholeskyQR2, Householder TSQR for the
        blocks it declines) or "householder" (TSQR every time); ``replace_every``: with
        ``one_reduction``, form Q = A P and alpha = P^T Q directly after every m-th
        iteration (and after a non-positive pivot of the recursive alpha).
        """
        s = B.shape[1]
        if X is None:
            X = torch.zeros_like(B) if isinstance(B, torch.Tensor) else np.zeros_like(B)
        want = np.float32 if prec == "fp32" else np.float64
        for blk in (B, X):
            if _prec_of(blk) != (L.BK_FP32 if want is np.float32 else L.BK_FP64):
                raise TypeError(f"prec {prec!r} needs {want.__name__} blocks")
        o = L.default_opts()
        o.eta, o.restart = float(eta), int(restart)
        o.norm_mode = {"max": 0, "fro": 1}[norm]
        o.ortho = {"cgs2": 0, "mgs": 1, "localized": 2}[ortho]
        o.prec = _PREC[prec]
        o.ir_inner_tol, o.ir_max_outer, o.sync_every = float(ir_inner_tol), int(ir_max_outer), int(sync_every)
        o.profile = 1 if profile else 0
        o.subalgebra_p = 0 if p is None else int(p)
        o.precond = None if precond is None else precond.ptr.value
        o.one_reduction = 1 if one_reduction else 0
        o.qr_mode = {"cholqr2": 0, "householder": 1}[qr]
        o.replace_every = int(replace_every)
        forced_arr = None
        if forced_reortho is not None:
            forced_arr = (C.c_uint8 * max(1, len(forced_reortho)))(*[1 if f else 0 for f in forced_reortho])
            o.forced_reortho = C.cast(forced_arr, C.POINTER(C.c_uint8))
            o.n_forced = len(forced_reortho)
        info = L.bkrylov_info()
        relres = (C.c_double * s)()
        nh = max(1, int(maxit) + 1) if record else 0
        hist = (C.c_double * max(1, nh))()
        dec = (C.c_uint8 * max(1, nh))()
        info.relres = C.cast(relres, C.POINTER(C.c_double))
        if record:
            info.history = C.cast(hist, C.POINTER(C.c_double))
            info.decisions = C.cast(dec, C.POINTER(C.c_uint8))
            info.history_len = nh
        fn = {"bcg": self.lib.bkrylov_solve_bcg, "bbicgstab": self.lib.bkrylov_solve_bbicgstab,
              "bgmres": self.lib.bkrylov_solve_bgmres}[method]
        st = fn(self.h, A.ptr, s, C.c_void_p(_ptr(B)), C.c_void_p(_ptr(X)), float(tol), int(maxit), C.byref(o),
                C.byref(info))
        if st not in (L.BK_OK, L.BK_NOT_CONVERGED, L.BK_BREAKDOWN, L.BK_NONFINITE, L.BK_TIMEOUT):
            raise BkError(st, f"bkrylov_solve_{method}")
        nrec = min(info.iters if prec != "fp32_ir" else info.outer + 1, nh)
        res = SolveInfo(
            status=st, status_name=L.status_string(st), iters=info.iters, reorths=info.reorths,
            converged=bool(info.converged), outer=info.outer, relres_max=info.relres_max,
            relres=np.array(relres[:s]), history=list(hist[:nrec]) if record else [],
            decisions=[bool(d) for d in dec[:nrec]] if record and prec != "fp32_ir" else [],
            elapsed_ms=info.elapsed_ms, reorths_cholqr=info.reorths_cholqr, replacements=info.replacements)
        return X, res


@dataclass
class SolveInfo:
    status: int
    status_name: str
    iters: int
    reorths: int
    converged: bool
    outer: int
    relres_max: float
    relres: np.ndarray
    history: list = field(default_factory=list)
    decisions: list = field(default_factory=list)
    elapsed_ms: float = 0.0
    reorths_cholqr: int = 0          # re-orthonormalisations done by CholeskyQR2
    replacements: int = 0            # 1R-BCG: direct recomputations of Q and alpha


class Operator:
    def __init__(self, h: Handle, ptr: C.c_void_p, n: int, keep=(), kind="csr", grid=None):
        self.h, self.ptr, self.n, self.keep, self.kind, self.grid = h, ptr, n, keep, kind, grid
        nn, nz = C.c_int64(), C.c_int64()
        _check(h.lib.bkrylov_op_size(ptr, C.byref(nn), C.byref(nz)), "bkrylov_op_size")
        self.nnz = nz.value

    def close(self):
        """Destroy the operator (idempotent) and drop the handle's reference to it."""
        if self.ptr:
            self.h.lib.bkrylov_op_destroy(self.ptr)
            self.ptr = None
        if self in self.h._ops:
            self.h._ops.remove(self)


def operator_from_problem(h: Handle, prob, use: str = "stencil", device="cuda") -> Operator:
    """Upload a ``workloads.Problem`` as a CSR or matrix-free stencil operator."""
    if use == "csr":
        A = prob.A
        return h.op_csr(torch.from_numpy(A.row_ptr).to(device), torch.from_numpy(A.col).to(device),
                        torch.from_numpy(A.val).to(device))
    st = prob.stencil
    if st["kind"] == "const7":
        return h.op_stencil("const7", st["nx"], st["ny"], st["nz"], st["coeffs"])
    if st["kind"] == "var7":
        k = torch.from_numpy(np.ascontiguousarray(st["k"], dtype=np.float64)).to(device)
        return h.op_stencil("var7", st["nx"], st["ny"], st["nz"], k)
    if st["kind"] == "edge5":
        e = np.concatenate([st["ax"].ravel(), st["ay"].ravel()])
        return h.op_stencil("edge5", st["nx"], st["ny"], 1, torch.from_numpy(e).to(device))
    raise KeyError(st["kind"])
