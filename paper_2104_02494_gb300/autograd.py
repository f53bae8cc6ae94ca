"""Differentiable block solve X = A(theta)^{-1} B with a hand-written adjoint.

Forward: block CG (FP64, or FP32 inner solves with FP64 refinement) on the
operator built from the parameters.  Backward, for G = dL/dX:
    A^T Lambda = G              (the same block solver; A is symmetric here)
    dL/dB = Lambda
    dL/da_ij = -sum_k Lambda_ik X_jk      on the sparsity pattern (CSR scatter kernel)
    dL/dtheta_e = a_e dL/da_e             for the per-edge model a_e = exp(theta_e)
                                          (edge kernel, chain rule included).
All products run in the library's kernels; torch only holds the tensors.
"""
from __future__ import annotations

import math

import torch

from .api import Handle


class BKrylovSolve(torch.autograd.Function):
    """X = solve(A, B) for a symmetric positive definite operator.

    params: either the CSR values (kind "csr", with the pattern in ``spec``)
    or the edge log-coefficients theta (kind "edge5", a_e = exp(theta_e)).
    spec: dict(kind=..., handle=Handle, and row_ptr/col (csr) or nx/ny (edge5),
    solve=dict of solver options).
    """

    @staticmethod
    def forward(ctx, params: torch.Tensor, B: torch.Tensor, spec: dict):
        h: Handle = spec["handle"]
        kind = spec["kind"]
        opts = dict(tol=1e-10, maxit=5000, eta=math.inf)
        opts.update(spec.get("solve", {}))
        p = params.detach().contiguous()
        if kind == "csr":
            op = h.op_csr(spec["row_ptr"], spec["col"], p)
        elif kind == "edge5":
            a = torch.exp(p)
            op = h.op_stencil("edge5", spec["nx"], spec["ny"], 1, a)
        else:
            raise KeyError(kind)
        X = torch.zeros_like(B)
        X, info = h.solve("bcg", op, B.detach().contiguous(), X, **opts)
        if not info.converged:
            raise RuntimeError(f"forward solve did not converge: {info.status_name}")
        ctx.spec, ctx.opts, ctx.op = spec, opts, op
        ctx.save_for_backward(X)
        return X

    @staticmethod
    def backward(ctx, G: torch.Tensor):
        (X,) = ctx.saved_tensors
        h: Handle = ctx.spec["handle"]
        op = ctx.op
        Lam = torch.zeros_like(X)
        Lam, info = h.solve("bcg", op, G.contiguous(), Lam, **ctx.opts)
        if not info.converged:
            raise RuntimeError(f"adjoint solve did not converge: {info.status_name}")
        if ctx.spec["kind"] == "csr":
            gp = h.adjoint_scatter(op, Lam, X)
        else:
            gp = h.edge_theta_grad(op, Lam, X)
        op.close()
        h._ops.remove(op)
        return gp, Lam, None
