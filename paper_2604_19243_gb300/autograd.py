"""torch.autograd wrapper of the FMM: phi = A(x) q with a hand-written backward.

Backward, for a loss L(phi) with g = dL/dphi and the tree held fixed:
  dL/dq   = A^T g                                   (the transposed FMM pass, fmm_adjoint)
  dL/dx_k = g_k grad phi_q(x_k) + q_k grad phi_g(x_k)
where phi_q, phi_g are the fields of densities q and g.  The second line is the derivative of
the exact kernel sum sum_i g_i sum_j K(x_i, x_j) q_j with respect to x_k, evaluated with the
FMM's gradients; it is the reading used for positions because the FMM's own map is only
piecewise smooth in x (boxes move with the points).
"""
from __future__ import annotations

import torch


class FmmFunction(torch.autograd.Function):
    """phi = FmmFunction.apply(q, x, fmm); `fmm` must hold a tree built over x."""

    @staticmethod
    def forward(ctx, q, x, fmm):
        need_grad_x = ctx.needs_input_grad[1]
        phi, grad = fmm.evaluate(q, gradient=need_grad_x)
        ctx.fmm = fmm
        if need_grad_x:
            ctx.save_for_backward(q, grad)
        else:
            ctx.save_for_backward(q)
        return phi

    @staticmethod
    def backward(ctx, g):
        fmm = ctx.fmm
        need_q, need_x = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        g = g.contiguous()
        psi, grad_g = fmm.adjoint(g, gradient=need_x)
        dq = psi.to(g.dtype) if need_q else None
        dx = None
        if need_x:
            q, grad_q = ctx.saved_tensors
            dx = g[:, None] * grad_q + q.to(g.dtype)[:, None] * grad_g
        return dq, dx, None


def fmm_energy(q, x, fmm):
    """E = 1/2 q . phi(q) with phi from the FMM (differentiable in q and x)."""
    return 0.5 * torch.dot(q, FmmFunction.apply(q, x, fmm))
