"""torch.autograd.Function wrappers around the C ABI.

HologramLoss (Sec. 3.2 L_MSE through Algorithms 2 and 3): the forward runs raster ->
BLASM -> loss and keeps only the parameters (no field, spectrum or intensity is
stored); the backward recomputes the forward inside the fused step (cgh_step_scaled) and
returns the parameter gradients -- the recompute-instead-of-store trade of the paper's
constant-VRAM backward.  The upstream gradient is applied inside the library's gradient
kernel, and the per-tile Gaussian lists the forward left in the plan's workspace are
reused when no other call on the plan has rebinned since (the saved parameters cannot
have changed: autograd rejects in-place changes to them).  With eager=True the forward already runs the fused step and keeps the
O(N) parameter gradients instead (no recompute; still no per-pixel state).

HologramIntensity returns I_l = |U(d_l)|^2 [L, C, H, W] for user-defined losses; its
backward recomputes the field and chains dL/dI through the intensity adjoint
(cgh_intensity_bwd), the adjoint propagation and the raster backward.  Every arithmetic
step of both runs in the library's kernels; this module only orders the calls.
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
            # the workspace now holds the binning of these parameters; autograd's version
            # check guarantees their values are unchanged when backward runs, so backward
            # may reuse it if no other call on the plan has rebinned in between
            ctx.bin_generation = plan.bin_generation
        return loss.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        plan = ctx.plan
        if ctx.eager:
            # chain rule with the upstream scalar (1 for loss.backward())
            grads = [g.mul_(grad_out) for g in ctx.saved_tensors]
        else:
            target, *ps = ctx.saved_tensors
            reuse = plan.bin_generation == ctx.bin_generation
            scale = grad_out.detach().reshape(1).to(torch.float32).contiguous()
            # the recomputed forward and the backward in one call; the upstream scalar is
            # applied inside the gradient kernel
            _, g = plan.step(dict(zip(PARAM_KEYS, ps)), target, grad_scale=scale,
                             reuse_binning=reuse)
            grads = [g[k] for k in PARAM_KEYS]
        return (None, None, None, *grads)


def hologram_loss(plan: Plan, params: dict, target: torch.Tensor, eager: bool = False):
    return HologramLoss.apply(plan, target, eager, *[params[k] for k in PARAM_KEYS])


class HologramIntensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan: Plan, *tensors):
        p = _params(tensors)
        ctx.plan = plan
        ctx.save_for_backward(*[p[k] for k in PARAM_KEYS])
        return plan.intensity(plan.blasm_fwd(plan.raster_fwd(p)))

    @staticmethod
    def backward(ctx, dI):
        plan = ctx.plan
        p = dict(zip(PARAM_KEYS, ctx.saved_tensors))
        Ud = plan.blasm_fwd(plan.raster_fwd(p))
        dUd = plan.intensity_bwd(Ud, dI.to(torch.float32).contiguous())
        g = plan.raster_bwd(p, plan.blasm_bwd(dUd))
        return (None, *[g[k] for k in PARAM_KEYS])


def hologram_intensity(plan: Plan, params: dict):
    return HologramIntensity.apply(plan, *[params[k] for k in PARAM_KEYS])
