"""Learned initialiser: a convolutional encoder that predicts Gaussian parameters from a
target intensity, trained on parameter sets produced by the plain optimiser.

The paper has no learned part; it names feed-forward prediction of the Gaussians as future
work (Sec. 6).  The encoder here is four 3x3 stride-2 convolutions, C -> 32 -> 64 -> 128 ->
S*(6+2C) channels with ReLU between them, so an H x W target becomes (H/16) x (W/16) cells
of S Gaussians each (512 x 512 RGB: 32 x 32 cells x 16 = 16,384 Gaussians).  Weights and
activations are BF16 with FP32 accumulation (cgh_conv3x3_fwd/bwd); FP32 master weights are
updated by the library's table-Adam and re-cast to BF16 after each step.  The last layer's
channels are decoded (cgh_encoder_decode) into offsets around per-slot anchors, so an
all-zero output is the structured initialisation with every Gaussian at its slot centre.

Training data come from the plain method itself: each target is optimised from that
anchor initialisation with Adam at the paper's learning rates (Sec. 4) through the
library's batched fused step, so every slot's optimised parameters stay attached to the
slot the encoder predicts for.  The training loss is the intensity loss of the decoded
prediction (Sec. 3.2, gradients from the library's raster + BLASM backward) plus a weighted
squared error to the optimiser's parameters.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import cgh, inputs
from .optim import LRS, HologramSet

WIDTHS = (32, 64, 128)
STRIDE = 2


class Encoder:
    """Weights, optimiser state and the forward/backward launch sequence of the encoder."""

    def __init__(self, C: int = 3, S: int = 16, widths: Sequence[int] = WIDTHS, device="cuda",
                 seed: int = 0, lr: float = 1e-3):
        self.C, self.S = C, S
        self.P = 6 + 2 * C
        self.chans = (C,) + tuple(widths) + (S * self.P,)
        self.device = device
        g = torch.Generator().manual_seed(seed)
        self.w, self.b, self.wb, self.dw, self.db = [], [], [], [], []
        groups = []
        n_layers = len(self.chans) - 1
        for i in range(n_layers):
            ci, co = self.chans[i], self.chans[i + 1]
            # He initialisation for the ReLU layers; a small last layer so that the first
            # predictions sit next to the anchors
            std = math.sqrt(2.0 / (9 * ci)) if i < n_layers - 1 else 1e-3
            w = (torch.randn(co, ci, 3, 3, generator=g) * std).to(device)
            b = torch.zeros(co, device=device)
            self.w.append(w)
            self.b.append(b)
            self.wb.append(torch.empty(co, ci, 3, 3, dtype=torch.bfloat16, device=device))
            self.dw.append(torch.zeros_like(w))
            self.db.append(torch.zeros_like(b))
            for p, gr in ((w, self.dw[-1]), (b, self.db[-1])):
                groups.append((p, torch.zeros_like(p), torch.zeros_like(p), gr, lr))
        self.adam = cgh.AdamTable(groups)
        self.sync_bf16()

    @property
    def n_layers(self) -> int:
        return len(self.w)

    def cells(self, H: int, W: int):
        cy, cx = H, W
        for _ in range(self.n_layers):
            cy, cx = cgh.conv_out_size(cy, STRIDE), cgh.conv_out_size(cx, STRIDE)
        return cy, cx

    def gaussians(self, H: int, W: int) -> int:
        cy, cx = self.cells(H, W)
        return cy * cx * self.S

    def sync_bf16(self):
        for w, wb in zip(self.w, self.wb):
            cgh.cast_bf16(w, wb)

    # ---------------------------------------------------------------- forward / backward
    def forward(self, target: torch.Tensor):
        """target [B, C, H, W] f32 intensity -> (output [B, S*P, CY, CX] f32, activations)."""
        x = cgh.cast_bf16(target.contiguous())
        acts = [x]
        for i in range(self.n_layers):
            last = i == self.n_layers - 1
            x = cgh.conv3x3_fwd(x, self.wb[i], self.b[i], STRIDE, relu=not last, out_f32=last)
            acts.append(x)
        return x, acts

    def backward(self, acts: List[torch.Tensor], dout: torch.Tensor):
        """Fills self.dw / self.db with the gradients for dL/d(output) = dout."""
        dy = dout
        for i in reversed(range(self.n_layers)):
            last = i == self.n_layers - 1
            dx, _, _ = cgh.conv3x3_bwd(acts[i], self.wb[i], acts[i + 1], dy, STRIDE,
                                       relu=not last, want_dx=i > 0, dw=self.dw[i],
                                       db=self.db[i])
            dy = dx

    def step(self):
        self.adam.step()
        self.sync_bf16()

    def predict(self, target: torch.Tensor, params: Optional[Dict[str, torch.Tensor]] = None):
        """Pre-activation parameters of B*N Gaussians for targets [B, C, H, W]."""
        out, _ = self.forward(target)
        H, W = target.shape[-2:]
        return cgh.encoder_decode(out, self.S, self.C, H, W, params=params)

    def anchors(self, B: int, H: int, W: int, params=None):
        """The structured initialisation: the decode of an all-zero encoder output."""
        cy, cx = self.cells(H, W)
        zero = torch.zeros(B, self.S * self.P, cy, cx, device=self.device)
        return cgh.encoder_decode(zero, self.S, self.C, H, W, params=params)

    def state_dict(self) -> Dict[str, np.ndarray]:
        d = {}
        for i in range(self.n_layers):
            d[f"w{i}"] = self.w[i].cpu().numpy()
            d[f"b{i}"] = self.b[i].cpu().numpy()
        return d

    def load_state_dict(self, d):
        for i in range(self.n_layers):
            self.w[i].copy_(torch.as_tensor(np.asarray(d[f"w{i}"])))
            self.b[i].copy_(torch.as_tensor(np.asarray(d[f"b{i}"])))
        self.sync_bf16()


# ------------------------------------------------------------------------- the workload
def planted_targets(count: int, H: int, W: int, wavelengths_m, pitch_m: float, z_m: float,
                    n_planted: int, seed: int, device, mean_intensity: float = 0.35):
    """[count, C, H, W] target intensities of structured planted scenes
    (inputs.planted_scene), rendered and propagated by the library to one plane at z_m,
    amplitudes scaled so that the mean intensity is `mean_intensity`, then clipped to
    [0, 1] (the displayable range the PSNR is taken on)."""
    C = len(wavelengths_m)
    plan = cgh.Plan(H, W, wavelengths_m, pitch_m, (z_m,), max_gaussians=n_planted, device=device)
    out = torch.empty(count, C, H, W, device=device)
    for i in range(count):
        p = {k: torch.from_numpy(v).to(device)
             for k, v in inputs.planted_scene(n_planted, C, H, W, seed + i).items()}
        I = plan.intensity(plan.blasm_fwd(plan.raster_fwd(p)))[0]
        I.mul_(mean_intensity / float(I.mean().clamp_min(1e-12)))
        out[i] = I.clamp_(0.0, 1.0)
    plan.close()
    return out


def psnr_db(loss: torch.Tensor) -> torch.Tensor:
    """PSNR (peak 1) from the intensity MSE."""
    return 10.0 * torch.log10(1.0 / loss.clamp_min(1e-12))


class Pipeline:
    """Data generation, training and evaluation of the learned initialiser for one image
    shape, on one plane.  `chunk` holograms are stepped together through one HologramSet."""

    def __init__(self, H: int, W: int, wavelengths_m=(638e-9, 520e-9, 450e-9), pitch_m=8e-6,
                 z_m: float = 5e-3, S: int = 16, chunk: int = 50, train_batch: int = 16,
                 device="cuda", seed: int = 0, lr: float = 1e-3):
        self.H, self.W = H, W
        self.wl, self.pitch, self.z = tuple(wavelengths_m), pitch_m, z_m
        self.C = len(self.wl)
        self.device = device
        self.enc = Encoder(self.C, S, device=device, seed=seed, lr=lr)
        self.N = self.enc.gaussians(H, W)
        self.chunk, self.train_batch = chunk, train_batch
        self._opt = None
        self._trainset = None

    def _optimiser_set(self) -> HologramSet:
        if self._opt is None:
            self._opt = HologramSet(self.chunk, self.H, self.W, self.wl, self.pitch, (self.z,),
                                    self.N, self.device)
        return self._opt

    def _train_set(self) -> HologramSet:
        if self._trainset is None:
            self._trainset = HologramSet(self.train_batch, self.H, self.W, self.wl, self.pitch,
                                         (self.z,), self.N, self.device)
        return self._trainset

    def _chunks(self, count: int):
        for s in range(0, count, self.chunk):
            yield s, min(self.chunk, count - s)

    def refine(self, init: Dict[str, torch.Tensor], targets: torch.Tensor, iters: int,
               warmup: int = 0):
        """Plain Adam from `init` ([M*N, ...] per group) on targets [M, C, H, W], learning
        rates ramped up over `warmup` iterations; returns (final parameters, loss history
        [M, iters+1])."""
        M = targets.shape[0]
        hs = self._optimiser_set()
        N = self.N
        final = {k: torch.empty_like(v) for k, v in init.items()}
        hist = torch.zeros(M, iters + 1, device=self.device)
        for s, n in self._chunks(M):
            sl = slice(s * N, (s + n) * N)
            padded = {k: torch.cat([v[sl], hs.params[k][n * N:]]) if n < self.chunk else v[sl]
                      for k, v in init.items()}
            tgt = targets[s:s + n].unsqueeze(1)
            if n < self.chunk:
                tgt = torch.cat([tgt, hs.targets[n:]])
            hs.load(padded, tgt)
            h = torch.zeros(self.chunk, iters + 1, device=self.device)
            hs.optimise(iters, h, warmup)
            hist[s:s + n] = h[:n]
            for k in final:
                final[k][sl] = hs.params[k][:n * N]
        return final, hist

    def generate(self, targets: torch.Tensor, iters: int, warmup: int = 0):
        """Training pairs: the plain optimiser's parameters for each target, started from the
        anchor initialisation."""
        init = self.enc.anchors(targets.shape[0], self.H, self.W)
        return self.refine(init, targets, iters, warmup)

    def train(self, targets: torch.Tensor, data: Dict[str, torch.Tensor], steps: int,
              param_weight: float = 1.0, render: bool = True, seed: int = 0,
              log_every: int = 0) -> List[tuple]:
        """`steps` minibatch steps.  Loss per image = intensity loss of the decoded
        prediction (if `render`) + param_weight * the mean over each parameter group of the
        squared error to the optimiser's parameters, summed over groups.  Returns
        (step, mean intensity loss, mean parameter term) every `log_every` steps."""
        M = targets.shape[0]
        B, N = self.train_batch, self.N
        ts = self._train_set()
        gen = torch.Generator(device="cpu").manual_seed(seed)
        cy, cx = self.enc.cells(self.H, self.W)
        ref = {k: torch.empty_like(v) for k, v in ts.params.items()}
        dout = torch.empty(B, self.enc.S * self.enc.P, cy, cx, device=self.device)
        pl = torch.zeros(1, device=self.device)
        log = []
        for it in range(steps):
            idx = torch.randint(0, M, (B,), generator=gen).to(self.device)
            ts.targets.copy_(targets.index_select(0, idx).unsqueeze(1))
            rows = (idx[:, None] * N + torch.arange(N, device=self.device)[None, :]).reshape(-1)
            for k in ref:
                ref[k].copy_(data[k].index_select(0, rows))
            out, acts = self.enc.forward(ts.targets[:, 0])
            cgh.encoder_decode(out, self.enc.S, self.C, self.H, self.W, params=ts.params)
            if render:
                ts.step_grads()
            pl.zero_()
            for k in cgh.PARAM_KEYS:
                cgh.mse_grad(ts.params[k], ref[k], param_weight / ref[k].numel() * B,
                             ts.grads[k], accumulate=render, loss_accum=pl)
            cgh.encoder_decode_bwd(ts.grads, B, cy, cx, self.enc.S, self.C, self.H, self.W,
                                   dout=dout)
            self.enc.backward(acts, dout)
            self.enc.step()
            if log_every and (it % log_every == 0 or it == steps - 1):
                img = float(ts.losses.mean()) if render else 0.0
                log.append((it, img, float(pl) / B))
        return log

    def predict(self, targets: torch.Tensor) -> Dict[str, torch.Tensor]:
        M = targets.shape[0]
        out = cgh.param_dict(M * self.N, self.C, self.device)
        for s in range(0, M, self.train_batch):
            n = min(self.train_batch, M - s)
            p = self.enc.predict(targets[s:s + n])
            for k in out:
                out[k][s * self.N:(s + n) * self.N] = p[k]
        return out

    def random_init(self, M: int, seed: int):
        """The plain method's initialisation (Sec. 4): uniform means, the workload's scale
        range, U(0,1) amplitudes, zero phases, opacity pre-activation -0.5."""
        out = cgh.param_dict(M * self.N, self.C, self.device)
        for i in range(M):
            p = inputs.gaussian_params(self.N, self.C, self.H, self.W, seed + i)
            p["phase"][:] = 0.0
            for k in out:
                out[k][i * self.N:(i + 1) * self.N] = torch.from_numpy(p[k]).to(self.device)
        return out

    def close(self):
        for s in (self._opt, self._trainset):
            if s is not None:
                s.close()


def iterations_to(hist_db: torch.Tensor, level: float):
    """Per image: first iteration whose PSNR reaches `level` dB (None if never)."""
    ok = hist_db >= level
    first = torch.where(ok.any(dim=1), ok.float().argmax(dim=1),
                        torch.full((hist_db.shape[0],), -1, device=hist_db.device))
    return [int(v) if v >= 0 else None for v in first.tolist()]
