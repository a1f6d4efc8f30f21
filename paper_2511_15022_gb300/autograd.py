"""torch.autograd.Function wrappers around the C ABI.

HologramLoss (Sec. 3.2 L_MSE through Algorithms 2 and 3): the forward runs raster ->
BLASM -> loss and keeps only the parameters (no field, spectrum or intensity is
stored); the backward recomputes the forward inside the fused cgh_step and returns the
parameter gradients -- the recompute-instead-of-store trade of the paper's constant-VRAM
backward.  With eager=True the forward already runs the fused step and keeps the
O(N) parameter gradients instead (no recompute; still no per-pixel state).

HologramIntensity returns I_l = |U(d_l)|^2 [L, C, H, W] for user-defined losses; its
backward recomputes the field and chains dL/dI through the adjoint propagation and the
raster backward.
"""
from __future__ import annotations

import torch

from .cgh import PARAM_KEYS, Plan


def _params(tensors):
    return {k: t.detach().contiguous() for k, t in zip(PARAM_KEYS, tensors)}


class HologramLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan: Plan, target: torch.Tensor, eager: bool, *tensors):
        p = _params(tensors)
        ctx.plan = plan
        ctx.eager = eager
        if eager:
            loss, grads = plan.step(p, target)
            ctx.save_for_backward(*[grads[k] for k in PARAM_KEYS])
        else:
            loss = plan.forward_loss(p, target)
            ctx.save_for_backward(target, *[p[k] for k in PARAM_KEYS])
        return loss.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        plan = ctx.plan
        if ctx.eager:
            grads = list(ctx.saved_tensors)
        else:
            target, *ps = ctx.saved_tensors
            _, g = plan.step(dict(zip(PARAM_KEYS, ps)), target)
            grads = [g[k] for k in PARAM_KEYS]
        # chain rule with the upstream scalar (1 for loss.backward())
        grads = [g.mul_(grad_out) for g in grads]
        return (None, None, None, *grads)


def hologram_loss(plan: Plan, params: dict, target: torch.Tensor, eager: bool = False):
    return HologramLoss.apply(plan, target, eager, *[params[k] for k in PARAM_KEYS])


class HologramIntensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan: Plan, *tensors):
        p = _params(tensors)
        ctx.plan = plan
        ctx.save_for_backward(*[p[k] for k in PARAM_KEYS])
        Ud = plan.blasm_fwd(plan.raster_fwd(p))
        return Ud.abs().square()

    @staticmethod
    def backward(ctx, dI):
        plan = ctx.plan
        p = dict(zip(PARAM_KEYS, ctx.saved_tensors))
        Ud = plan.blasm_fwd(plan.raster_fwd(p))
        dUd = (2.0 * dI.contiguous()) * Ud  # dL/dRe + j dL/dIm = 2 dL/dI U
        g = plan.raster_bwd(p, plan.blasm_bwd(dUd.contiguous()))
        return (None, *[g[k] for k in PARAM_KEYS])


def hologram_intensity(plan: Plan, params: dict):
    return HologramIntensity.apply(plan, *[params[k] for k in PARAM_KEYS])
