"""Differentiable block solve X = A(theta)^{-1} B with a hand-written adjoint.

Forward: a block solver of the library (block CG by default, FP64 or FP32 inner
solves with FP64 refinement) on the operator built from the parameters.
Backward, for G = dL/dX:
    A^T Lambda = G              (the same block solver on the transposed operator)
    dL/dB = Lambda
    dL/da_ij = -sum_k Lambda_ik X_jk      on the sparsity pattern (CSR scatter kernel)
    dL/dtheta_e = a_e dL/da_e             for the per-edge model a_e = exp(theta_e)
                                          (edge kernel, chain rule included).
The operator, exp(theta), the transpose, the solves and the gradients are all
formed by the library; this module only passes tensors.  Each of forward and
backward builds its own operator and destroys it before returning, so nothing
stays allocated when backward never runs (no_grad, inference) or runs twice.
"""
from __future__ import annotations

import math

import torch

from .api import Handle


def _operator(h: Handle, spec: dict, p: torch.Tensor):
    kind = spec["kind"]
    if kind == "csr":
        return h.op_csr(spec["row_ptr"], spec["col"], p)
    if kind == "edge5":
        return h.op_stencil("edge5_log", spec["nx"], spec["ny"], 1, p)
    raise KeyError(kind)


class BKrylovSolve(torch.autograd.Function):
    """X = solve(A(params), B).

    params: either the CSR values (kind "csr", with the pattern in ``spec``)
    or the edge log-coefficients theta (kind "edge5", a_e = exp(theta_e)).
    spec: dict(kind=..., handle=Handle, and row_ptr/col (csr) or nx/ny (edge5),
    method="bcg" (default; A symmetric positive definite), "bbicgstab" or "bgmres"
    (a non-symmetric A), solve=dict of solver options).  The adjoint solve runs the
    same method on A^T (for kind "csr" a transposed operator formed on the device;
    the per-edge operator is symmetric).
    """

    @staticmethod
    def forward(ctx, params: torch.Tensor, B: torch.Tensor, spec: dict):
        h: Handle = spec["handle"]
        method = spec.get("method", "bcg")
        opts = dict(tol=1e-10, maxit=5000, eta=math.inf)
        opts.update(spec.get("solve", {}))
        p = params.detach().contiguous()
        op = _operator(h, spec, p)
        try:
            X = torch.zeros_like(B)
            X, info = h.solve(method, op, B.detach().contiguous(), X, **opts)
        finally:
            op.close()
        if not info.converged:
            raise RuntimeError(f"forward solve did not converge: {info.status_name}")
        ctx.spec, ctx.opts, ctx.method = spec, opts, method
        ctx.save_for_backward(p, X)
        return X

    @staticmethod
    def backward(ctx, G: torch.Tensor):
        p, X = ctx.saved_tensors
        h: Handle = ctx.spec["handle"]
        csr = ctx.spec["kind"] == "csr"
        op = _operator(h, ctx.spec, p)
        opT = None
        try:
            opT = h.op_transpose(op) if csr else op
            Lam = torch.zeros_like(X)
            Lam, info = h.solve(ctx.method, opT, G.contiguous(), Lam, **ctx.opts)
            if not info.converged:
                raise RuntimeError(f"adjoint solve did not converge: {info.status_name}")
            gp = h.adjoint_scatter(op, Lam, X) if csr else h.edge_theta_grad(op, Lam, X)
        finally:
            if opT is not None and opT is not op:
                opT.close()
            op.close()
        return gp, Lam, None
