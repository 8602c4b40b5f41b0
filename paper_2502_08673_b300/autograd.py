"""torch.autograd.Function over the relaxed circuit.

forward(V) runs sat_forward (Eqs. 5-7) and returns the per-sample loss;
backward runs the hand-written adjoint sat_backward (Eq. 8, Table 1
derivatives).  V is [n_pi, B] float32 on the current CUDA device.
"""
from __future__ import annotations

import torch

from . import api


class CircuitLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, plan, act_dtype="f32"):
        V = V.contiguous()
        B = V.shape[1]
        act = api.new_act(plan, B, act_dtype, V.device)
        loss = torch.empty(B, dtype=torch.float32, device=V.device)
        api.sat_forward(plan, V, act, loss, act_dtype)
        ctx.save_for_backward(V, act)
        ctx.plan, ctx.act_dtype = plan, act_dtype
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        V, act = ctx.saved_tensors
        B = V.shape[1]
        adj = api.new_adj(ctx.plan, B, V.device)
        gV = torch.zeros_like(V)
        api.sat_backward(ctx.plan, V, act, adj, gV, grad_loss.contiguous().float(), ctx.act_dtype)
        return gV, None, None


def circuit_loss(V, plan, act_dtype="f32"):
    """Per-sample l2 loss of the relaxed circuit, differentiable w.r.t. V."""
    return CircuitLoss.apply(V, plan, act_dtype)
