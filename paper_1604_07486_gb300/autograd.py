"""Differentiable conversion: a torch.autograd.Function whose backward applies A^T.

beta = A alpha is linear, so d(loss)/d(alpha) = A^T d(loss)/d(beta).  The forward pass calls
tdh_plan_execute and the backward pass tdh_plan_execute_adjoint (same plan: A^T =
D2 (T^T o H) D1 with H symmetric, the Toeplitz part applied with the conjugate symbol).
"""
import torch


class _Convert(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alpha, plan):
        ctx.plan = plan
        return plan.execute(alpha.contiguous())

    @staticmethod
    def backward(ctx, grad_beta):
        return ctx.plan.adjoint(grad_beta.contiguous()), None


def convert(alpha, plan):
    """beta = A alpha with gradients; alpha: CUDA tensor [..., n] of the plan's dtype."""
    return _Convert.apply(alpha, plan)
