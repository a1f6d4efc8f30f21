"""FP64 CPU oracle for the learned initialiser's layers.  TEST INFRASTRUCTURE ONLY (see
oracle/__init__.py for who may import it).

The paper has no learned part; it names feed-forward prediction of the Gaussians as future
work (Sec. 6).  The layers restated here are the workload's encoder: 3x3 convolutions with
zero padding 1 and a stride, ReLU, and the affine decode from the last layer's channels to
pre-activation Gaussian parameters around per-slot anchors.  Plain numpy, float64: the
convolution is its definition, one einsum per kernel tap over strided views of the padded
input.

Pinned by tests/test_oracle_encoder.py against torch.nn.functional.conv2d (CPU, float64)
and central finite differences of these functions.
"""
from __future__ import annotations

import numpy as np


def conv3x3_fwd(x, w, b, stride: int, relu: bool):
    """y[b,o,i,j] = act(bias[o] + sum_{c,ky,kx} w[o,c,ky,kx] x[b,c,i*s+ky-1,j*s+kx-1])."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    B, C, H, W = x.shape
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    y = np.zeros((B, w.shape[0], Ho, Wo)) + np.asarray(b, np.float64)[None, :, None, None]
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride]
            y += np.einsum("oc,bchw->bohw", w[:, :, ky, kx], patch)
    return np.maximum(y, 0.0) if relu else y


def conv3x3_bwd(x, w, y, dy, stride: int, relu: bool):
    """Gradients (dx, dw, db) of conv3x3_fwd given the output y and dL/dy."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    g = np.asarray(dy, np.float64) * ((np.asarray(y) > 0) if relu else 1.0)
    B, C, H, W = x.shape
    Ho, Wo = g.shape[2], g.shape[3]
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            sl = (slice(None), slice(None), slice(ky, ky + stride * (Ho - 1) + 1, stride),
                  slice(kx, kx + stride * (Wo - 1) + 1, stride))
            dw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", g, xp[sl])
            dxp[sl] += np.einsum("oc,bohw->bchw", w[:, :, ky, kx], g)
    return dxp[:, :, 1:H + 1, 1:W + 1], dw, g.sum(axis=(0, 2, 3))


POS_SCALE, SCALE_SCALE, S_BASE, AMP_BASE, AMP_SCALE, ALPHA_BASE = 0.02, 0.5, np.log(1.5), 0.5, 0.5, -0.5


def decode(out, S: int, C: int, H: int, W: int):
    """Encoder output [B, S*P, CY, CX] -> per-image parameter dicts (P = 6 + 2C)."""
    out = np.asarray(out, np.float64)
    B, _, CY, CX = out.shape
    P = 6 + 2 * C
    side = int(np.ceil(np.sqrt(S)))
    o = out.reshape(B, S, P, CY, CX).transpose(0, 3, 4, 1, 2).reshape(B, CY * CX * S, P)
    n = np.arange(CY * CX * S)
    cell, g = n // S, n % S
    cy, cx = cell // CX, cell % CX
    ax = (cx + ((g % side) + 0.5) / side) * (W / CX)
    ay = (cy + ((g // side) + 0.5) / side) * (H / CY)
    anx = np.arctanh(np.clip(2 * ax / W - 1, -0.999999, 0.999999))
    any_ = np.arctanh(np.clip(2 * ay / H - 1, -0.999999, 0.999999))
    res = []
    for b in range(B):
        ob = o[b]
        res.append({
            "xy_raw": np.stack([anx + POS_SCALE * ob[:, 0], any_ + POS_SCALE * ob[:, 1]], axis=1),
            "s_raw": S_BASE + SCALE_SCALE * ob[:, 2:4],
            "theta": ob[:, 4],
            "amp": AMP_BASE + AMP_SCALE * ob[:, 5:5 + C],
            "phase": ob[:, 5 + C:5 + 2 * C],
            "alpha_raw": ALPHA_BASE + ob[:, 5 + 2 * C],
        })
    return res


def decode_bwd(grads, S: int, C: int, CY: int, CX: int):
    """Adjoint of decode: per-image gradient dicts w.r.t. the decoded parameters ->
    dL/d(encoder output) [B, S*P, CY, CX].  The decode is affine, so each output channel's
    gradient is its parameter's gradient times the channel's scale."""
    P = 6 + 2 * C
    B = len(grads)
    o = np.zeros((B, CY * CX * S, P))
    for b, g in enumerate(grads):
        o[b, :, 0:2] = POS_SCALE * np.asarray(g["xy_raw"], np.float64)
        o[b, :, 2:4] = SCALE_SCALE * np.asarray(g["s_raw"], np.float64)
        o[b, :, 4] = np.asarray(g["theta"], np.float64)
        o[b, :, 5:5 + C] = AMP_SCALE * np.asarray(g["amp"], np.float64)
        o[b, :, 5 + C:5 + 2 * C] = np.asarray(g["phase"], np.float64)
        o[b, :, 5 + 2 * C] = np.asarray(g["alpha_raw"], np.float64)
    return o.reshape(B, CY, CX, S, P).transpose(0, 3, 4, 1, 2).reshape(B, S * P, CY, CX)
