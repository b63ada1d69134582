"""Differentiable solve: psi_h(F, psi0) with gradients by the adjoint solve.

psi = K^{-1} (F - m_t (x) A_x psi0) + 1 (x) psi0 is C-linear in (F, psi0), so with
PyTorch's complex convention (the gradient of a real loss w.r.t. z is dL/d(conj z),
and for a linear y = L x, grad_x = L^H grad_y):

    grad_F    = K^{-H} grad_psi                                   (st_adjoint_solve)
    grad_psi0 = sum_l grad_psi[l, :] - A_x (m_t^T grad_F)         (st_adjoint_lift)

K^H lambda = g is solved with the same time decomposition and the same spatial
factorisations as the forward solve (C_k is complex symmetric).
"""
from __future__ import annotations

import torch

from . import stfdm


class STSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, psi0, handle, precision="fp64", tol=0.0):
        ctx.handle = handle
        ctx.precision = precision
        ctx.tol = tol
        ctx.has_psi0 = psi0 is not None
        psi, _ = stfdm.st_fdm_solve(handle, F.contiguous(), psi0.contiguous() if psi0 is not None else None,
                                    precision=precision, tol=tol, want_info=False)
        return psi

    @staticmethod
    def backward(ctx, grad_psi):
        h = ctx.handle
        g = grad_psi.contiguous()
        if ctx.precision == "fp32":
            g = g.to(torch.complex64)
        grad_F, _ = stfdm.st_adjoint_solve(h, g, precision=ctx.precision, tol=ctx.tol, want_info=False)
        grad_psi0 = None
        if ctx.has_psi0 and ctx.needs_input_grad[1]:
            grad_psi0 = stfdm.st_adjoint_lift(h, grad_psi.to(torch.complex128).contiguous(),
                                              grad_F.to(torch.complex128).contiguous())
            if ctx.precision == "fp32":
                grad_psi0 = grad_psi0.to(torch.complex64)
        return grad_F, grad_psi0, None, None, None


def st_solve(F, psi0, handle, precision="fp64", tol=0.0):
    """Differentiable psi_h = solve(F, psi0) on the handle's problem."""
    return STSolve.apply(F, psi0, handle, precision, tol)
