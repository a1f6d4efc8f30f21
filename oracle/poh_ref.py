"""FP64 CPU oracle for the phase-only hologram (POH) conversion of Sec. 3.3.  TEST
INFRASTRUCTURE ONLY (see oracle/__init__.py for who may import it).

* Smooth POH by double-phase amplitude coding (DPAC, the method the paper cites): with
  A_n = |H| / max |H| per channel and phi = arg H, phi_DPAC = phi + acos(A_n) where i + j is
  even and phi - acos(A_n) where it is odd; H_smooth = exp(j phi_DPAC).  The formula the
  paper prints (A where i + j is even, phi where odd) is kept as mode "printed".
* Random POH: H_rand = exp(j phi_rand) with a learnable phase field phi_rand [C, H, W],
  propagated beside the Gaussians' field H; the joint objective is
    L_extract = sum_l [ R_l(I_l) + R_l(I_rand,l) + lambda_comp mean (I_l - I_rand,l)^2
                        + lambda_field mean (|Re(U_l - U_rand,l)| + |Im(U_l - U_rand,l)|) ]
  where R_l is plane l's part of L_recon (the three squared terms, mean over C, H, W) and
  every mean runs over the C x H x W values of one plane.
Plain numpy, float64; the propagation and rasterisation steps are the pinned oracle
functions of oracle/__init__.py.

Pinned by tests/test_oracle_poh.py: a closed form of the DPAC pattern's spectrum, the
decomposition of L_extract into the pinned L_recon and MSE oracles plus a complex L1 term
with an explicit sign gradient, and finite differences of the phase gradient and of the
whole conversion step.
"""
from __future__ import annotations

import numpy as np

import oracle


def dpac(Hf, mode: str = "double"):
    """Smooth POH of a complex field [C, H, W]: exp(j phi_DPAC) (Sec. 3.3).
    mode "double": double-phase amplitude coding, the method the paper cites -- with
    A_n = |H| / max|H| per channel and phi = arg H, phi_DPAC = phi + acos(A_n) where i + j
    is even and phi - acos(A_n) where it is odd (each neighbouring pair averages to
    A_n exp(j phi)).  mode "printed": the formula as printed, A where i + j is even and phi
    where it is odd."""
    Hf = np.asarray(Hf, np.complex128)
    C, H, W = Hf.shape
    A = np.abs(Hf)
    phi = np.angle(Hf)
    even = ((np.arange(H)[:, None] + np.arange(W)[None, :]) % 2) == 0
    if mode == "printed":
        pd = np.where(even[None], A, phi)
    else:
        amax = A.reshape(C, -1).max(axis=1)[:, None, None]
        a = np.arccos(np.clip(A / np.where(amax > 0, amax, 1.0), 0.0, 1.0))
        pd = np.where(even[None], phi + a, phi - a)
    return np.exp(1j * pd)


def poh_field(phi):
    """H_rand = exp(j phi_rand)."""
    return np.exp(1j * np.asarray(phi, np.float64))


def phase_grad(phi, dH):
    """dL/dphi from dH = dL/dRe + j dL/dIm of H_rand = exp(j phi):
    dRe/dphi = -sin phi, dIm/dphi = cos phi."""
    phi = np.asarray(phi, np.float64)
    dH = np.asarray(dH, np.complex128)
    return -np.sin(phi) * dH.real + np.cos(phi) * dH.imag


def extract_loss(Ud, Ud_rand, target, mask=None, lambda_comp=0.1, lambda_field=0.01):
    """L_extract over L planes; Ud, Ud_rand complex [L, C, H, W].  Returns (loss, dL/dUd,
    dL/dUd_rand), gradients as dRe + j dIm."""
    Ud = np.asarray(Ud, np.complex128)
    Ur = np.asarray(Ud_rand, np.complex128)
    T = np.asarray(target, np.float64)
    L = Ud.shape[0]
    n = Ud[0].size  # values per plane
    # the two L_recon terms: oracle.recon_loss averages over planes, here they are summed
    r1, g1 = oracle.recon_loss(Ud, T, mask)
    r2, g2 = oracle.recon_loss(Ur, T, mask)
    loss = L * (r1 + r2)
    dU = L * g1
    dR = L * g2
    I = np.abs(Ud) ** 2
    Ir = np.abs(Ur) ** 2
    dI = I - Ir
    loss += lambda_comp * np.sum(dI * dI) / n
    gI = 2.0 * lambda_comp * dI / n          # dL/dI; dL/dI_rand = -gI
    dU += gI * 2.0 * Ud
    dR += -gI * 2.0 * Ur
    D = Ud - Ur
    loss += lambda_field * np.sum(np.abs(D.real) + np.abs(D.imag)) / n
    gD = lambda_field * (np.sign(D.real) + 1j * np.sign(D.imag)) / n
    dU += gD
    dR -= gD
    return float(loss), dU, dR


def poh_step(params, phi, target, H, W, lambdas, pitch, z, pad=2, cutoff=1.0 / 255.0,
             mask=None, lambda_comp=0.1, lambda_field=0.01):
    """One joint forward + backward pass of the random-POH conversion: returns dict(loss,
    grads (Gaussian parameters), dphi)."""
    U0, Ud = oracle.forward(params, H, W, lambdas, pitch, z, pad, cutoff)
    Hr = poh_field(phi)
    Ur = oracle.blasm_fwd(Hr, lambdas, pitch, z, pad)
    loss, dU, dR = extract_loss(Ud, Ur, target, mask, lambda_comp, lambda_field)
    dU0 = oracle.blasm_bwd(dU, lambdas, pitch, z, pad)
    grads = oracle.raster_bwd(params, H, W, dU0, cutoff)
    dHr = oracle.blasm_bwd(dR, lambdas, pitch, z, pad)
    return {"loss": loss, "grads": grads, "dphi": phase_grad(phi, dHr)}
