"""Propagation parity for every specialised padded length: the batched workload's size
buckets (512x768, 640x1024, 1024x1024 images), the 1440x2560, 1800x3200 and 2160x3840
holograms, one channel and plane each against the oracle, plus specialised == generic
kernels on the same plan for every shape (including the 1080x1920 hologram the benchmark
times): the fused step runs both column kernels, the forward-model and the adjoint one,
whose radix orders may differ."""
import numpy as np
import pytest

import oracle
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import c64, rel_l2

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-4

SHAPES = [(512, 768), (640, 1024), (1024, 1024), (512, 512), (1440, 2560), (1800, 3200),
          (2160, 3840)]


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


@pytest.mark.parametrize("H,W", SHAPES)
def test_blasm_matches_oracle(H, W, dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    lam, z = 520e-9, 7e-3
    plan = cgh.Plan(H, W, (lam,), 8e-6, (z,), max_gaussians=1, device=dev)
    U0 = inputs.random_field(1, H, W, seed=H + W)
    Ud = c64(plan.blasm_fwd(torch.from_numpy(U0).to(dev)))
    ref = oracle.blasm_fwd(U0, [lam], 8e-6, [z])
    assert rel_l2(Ud, ref) < FIELD_TOL
    if H * W <= 1024 * 1024:
        dUd = inputs.random_field(1, H, W, seed=H + W + 1)[None]
        dU0 = c64(plan.blasm_bwd(torch.from_numpy(dUd).to(dev)))
        refb = oracle.blasm_bwd(dUd, [lam], 8e-6, [z])
        assert rel_l2(dU0, refb) < FIELD_TOL


@pytest.mark.parametrize("H,W", SHAPES + [(1080, 1920)])
def test_specialised_equals_generic(H, W, dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    w = inputs.custom(H, W, 3000, wavelengths_m=(638e-9, 450e-9), z_m=(0.0, 6e-3), seed=W)
    p = {k: torch.from_numpy(v).to(dev) for k, v in inputs.params_for(w).items()}
    t = torch.from_numpy(inputs.blob_targets(w.L, w.C, H, W)).to(dev)
    spec = cgh.Plan(H, W, w.wavelengths_m, w.pitch_m, w.z_m, max_gaussians=w.N, device=dev)
    gen = cgh.Plan(H, W, w.wavelengths_m, w.pitch_m, w.z_m, max_gaussians=w.N, device=dev,
                   tuning={"fft_kernels": 2})
    l1, g1 = spec.step(p, t)
    l2, g2 = gen.step(p, t)
    assert abs(l1.item() - l2.item()) < 1e-5 * l2.item()
    for k in g1:
        assert rel_l2(g1[k].cpu().numpy(), g2[k].cpu().numpy()) < 1e-4, k


def test_pad3_general_window(dev):
    """Pad factor 3 on a 720 x 1280 image gives the 2160 x 3840 padded grid of the 1080p
    hologram with the image window at a third of each length (rows 720..1439, columns
    1280..2559): the specialised kernels then run their general instantiations (window tested
    at run time per element, not resolved at compile time).  Forward and adjoint propagation
    against the oracle, and the fused step against the generic kernels."""
    import torch
    from paper_2511_15022_gb300 import cgh
    H, W, lam, z = 720, 1280, 520e-9, 7e-3
    plan = cgh.Plan(H, W, (lam,), 8e-6, (z,), pad=3, max_gaussians=1, device=dev)
    U0 = inputs.random_field(1, H, W, seed=33)
    Ud = c64(plan.blasm_fwd(torch.from_numpy(U0).to(dev)))
    assert rel_l2(Ud, oracle.blasm_fwd(U0, [lam], 8e-6, [z], pad=3)) < FIELD_TOL
    dUd = inputs.random_field(1, H, W, seed=34)[None]
    dU0 = c64(plan.blasm_bwd(torch.from_numpy(dUd).to(dev)))
    assert rel_l2(dU0, oracle.blasm_bwd(dUd, [lam], 8e-6, [z], pad=3)) < FIELD_TOL

    w = inputs.custom(H, W, 3000, wavelengths_m=(638e-9, 450e-9), z_m=(0.0, 6e-3), seed=35)
    p = {k: torch.from_numpy(v).to(dev) for k, v in inputs.params_for(w).items()}
    t = torch.from_numpy(inputs.blob_targets(w.L, w.C, H, W)).to(dev)
    spec = cgh.Plan(H, W, w.wavelengths_m, w.pitch_m, w.z_m, pad=3, max_gaussians=w.N,
                    device=dev)
    gen = cgh.Plan(H, W, w.wavelengths_m, w.pitch_m, w.z_m, pad=3, max_gaussians=w.N,
                   device=dev, tuning={"fft_kernels": 2})
    l1, g1 = spec.step(p, t)
    l2, g2 = gen.step(p, t)
    assert abs(l1.item() - l2.item()) < 1e-5 * l2.item()
    for k in g1:
        assert rel_l2(g1[k].cpu().numpy(), g2[k].cpu().numpy()) < 1e-4, k
