"""Differentiable structured random operator: z = A(theta) x as a torch.autograd.Function.

Forward and backward run in the CUDA library: the forward is sr_forward with
the phases theta (a trainable float32 tensor [L, m]) loaded into the plan's
diagonals on the device; the backward is sr_backward, which returns A^H G_z
and the phase gradient sum_b Im(conj(p_l) h_l) while recomputing the layer
inputs instead of storing them (Sec. III, Eq. 5 with D_l = diag(exp(i theta_l))).
"""
from __future__ import annotations

import torch

from .plan import Plan


class StructuredRandomOp(torch.autograd.Function):
    """z = A(theta) x. Usage: z = StructuredRandomOp.apply(x, theta, plan)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, theta: torch.Tensor, plan: Plan) -> torch.Tensor:
        plan.set_phases_device(theta.detach().to(torch.float32))
        x = x.detach().contiguous()
        ctx.plan = plan
        ctx.save_for_backward(x, theta)
        return plan.forward(x)

    @staticmethod
    def backward(ctx, gz: torch.Tensor):
        x, theta = ctx.saved_tensors
        plan = ctx.plan
        plan.set_phases_device(theta.detach().to(torch.float32))  # the plan may have been reused since
        gx, gth = plan.backward(x, gz.contiguous(), need_x=ctx.needs_input_grad[0],
                                need_theta=ctx.needs_input_grad[1])
        if gth is not None:
            gth = gth.to(theta.dtype)
        return gx, gth, None


def structured_random(x: torch.Tensor, theta: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Functional form of StructuredRandomOp."""
    return StructuredRandomOp.apply(x, theta, plan)
