"""Optimiser plumbing around the C ABI: the paper's per-group learning rates and a set of
same-shape holograms optimised together (one graph launch for all fused forward+backward
passes, one table-Adam launch for all parameters).

Every arithmetic step runs in the library's kernels; this module only allocates device
buffers, binds them and orders the launches.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import torch

from . import cgh

# Adam learning rates per parameter group (Sec. 4; the position rate is the start of the
# paper's cosine schedule, 1e-2 -> 1e-3)
LRS = {"xy_raw": 1e-2, "s_raw": 5e-3, "theta": 1e-3, "amp": 2.5e-3, "phase": 2.5e-3,
       "alpha_raw": 2.5e-2}


class HologramSet:
    """B holograms of one shape (H x W, C wavelengths, L planes, N Gaussians each).

    Parameters and gradients are stored as one array per group over all B*N Gaussians
    (hologram i owns rows i*N .. (i+1)*N), targets as [B, L, C, H, W] and losses as [B, 1].
    `step_grads()` runs every hologram's fused raster -> BLASM -> loss -> backward in one
    graph launch; `optimise()` adds one table-Adam launch per iteration."""

    def __init__(self, B: int, H: int, W: int, wavelengths_m: Sequence[float], pitch_m: float,
                 z_m: Sequence[float], N: int, device, lrs: Optional[Dict[str, float]] = None,
                 cutoff: float = 1.0 / 255.0):
        self.B, self.H, self.W, self.N = B, H, W, N
        self.C, self.L = len(wavelengths_m), len(z_m)
        self.device = device
        self.plans = [cgh.Plan(H, W, wavelengths_m, pitch_m, z_m, cutoff=cutoff, max_gaussians=N,
                               device=device) for _ in range(B)]
        self.params = cgh.param_dict(B * N, self.C, device)
        self.grads = cgh.param_dict(B * N, self.C, device)
        for d in (self.params, self.grads):
            for v in d.values():
                v.zero_()
        self.exp_avg = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.exp_avg_sq = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.targets = torch.zeros(B, self.L, self.C, H, W, device=device)
        self.losses = torch.zeros(B, 1, device=device)
        self.batch = cgh.Batch(self.plans)
        for i in range(B):
            self.batch.bind(i, self.slice(self.params, i), self.targets[i],
                            self.slice(self.grads, i), self.losses[i])
        lrs = lrs or LRS
        self.adam = cgh.AdamTable([(self.params[k], self.exp_avg[k], self.exp_avg_sq[k],
                                    self.grads[k], lrs[k]) for k in cgh.PARAM_KEYS])

    def slice(self, d: Dict[str, torch.Tensor], i: int) -> Dict[str, torch.Tensor]:
        return {k: v[i * self.N:(i + 1) * self.N] for k, v in d.items()}

    def load(self, params: Optional[Dict[str, torch.Tensor]] = None, targets=None):
        """Copy initial parameters ([B*N, ...] per group) and/or targets in, reset Adam."""
        if params is not None:
            for k in cgh.PARAM_KEYS:
                self.params[k].copy_(params[k].reshape(self.params[k].shape))
        if targets is not None:
            self.targets.copy_(targets.reshape(self.targets.shape))
        for k in cgh.PARAM_KEYS:
            self.exp_avg[k].zero_()
            self.exp_avg_sq[k].zero_()
        self.adam.t = 0

    def step_grads(self):
        """Loss and gradients of every hologram at the current parameters."""
        self.batch.step()

    def optimise(self, iters: int, history: Optional[torch.Tensor] = None, warmup: int = 0):
        """`iters` Adam iterations, learning rates ramped linearly over the first `warmup`.
        If given, history [B, >= iters+1] receives the loss before each update and, in its
        last column, the loss after the final update."""
        for it in range(iters):
            self.batch.step()
            if history is not None:
                history[:, it].copy_(self.losses[:, 0])
            self.adam.step(min(1.0, (it + 1) / warmup) if warmup > 0 else 1.0)
        if history is not None:
            self.batch.step()
            history[:, iters].copy_(self.losses[:, 0])

    def close(self):
        self.batch.close()
        for p in self.plans:
            p.close()
