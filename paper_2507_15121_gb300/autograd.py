"""Gradient-based CP completion on top of the CUDA library.

``CPSampled`` is a ``torch.autograd.Function`` whose forward evaluates the CP
model at the tensor's nonzeros (m_k = sum_r prod_n A_n(i_n(k), r), the CP
model of Sec. 2.1 sampled at the coordinates) and whose hand-written
backward is MTTKRP with the incoming per-nonzero gradient as the values:
dL/dA_n = MTTKRP_n(values = dL/dm) for every mode n.
"""
from __future__ import annotations

import torch

from .tensor import Tensor


class CPSampled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tensor: Tensor, *factors):
        ctx.tensor = tensor
        ctx.save_for_backward(*factors)
        return tensor.cp_sample(list(factors))

    @staticmethod
    def backward(ctx, grad_m):
        factors = ctx.saved_tensors
        grads = ctx.tensor.cp_grad(list(factors), grad_m.float().contiguous())
        grads = [g if g.dtype == f.dtype else g.to(f.dtype) for g, f in zip(grads, factors)]
        needs = ctx.needs_input_grad[1:]
        return (None, *[g if need else None for g, need in zip(grads, needs)])


class CPCompletionLoss(torch.autograd.Function):
    """L = 1/2 sum_k (m_k - x_k)^2 over the tensor's own values, as one fused
    pass per mode: the forward computes the loss and every factor gradient
    together (amped_cp_completion_grad); the backward scales the stored
    gradients by the incoming gradient of L."""

    @staticmethod
    def forward(ctx, tensor: Tensor, *factors):
        grads, loss = tensor.completion_grad(list(factors))
        ctx.save_for_backward(*grads)
        ctx.dtypes = [f.dtype for f in factors]
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        grads = ctx.saved_tensors
        out = [(g * grad_loss).to(dt) for g, dt in zip(grads, ctx.dtypes)]
        needs = ctx.needs_input_grad[1:]
        return (None, *[g if need else None for g, need in zip(out, needs)])


def fused_completion_loss(tensor: Tensor, factors):
    """1/2 sum_k (m_k - x_k)^2 over the tensor's stored values x, differentiable in
    the factors, computed by the fused kernels (one pass per mode)."""
    return CPCompletionLoss.apply(tensor, *factors)


def sampled_model(tensor: Tensor, factors):
    """m_k at every nonzero (caller order), differentiable in the factors."""
    return CPSampled.apply(tensor, *factors)


def completion_loss(tensor: Tensor, factors, x):
    """L = 1/2 sum_k (m_k - x_k)^2 over the observed entries x (caller order)."""
    m = sampled_model(tensor, factors)
    return 0.5 * torch.sum((m - x) ** 2)
