"""Planes at distance 0 (Algorithm 3 with d = 0: H = 1 on every bin when there is no
aperture, so U(d) = U(0)).  The fused step, the forward-only loss and the autograd function
take such planes' loss and gradient seed on U(0) in the pixel domain and propagate only the
others; with the tuning knob identity_planes = 2 every plane goes through the FFT passes.
Both must match the FP64 oracle, which propagates every plane with its textbook FFT, for
plane sets with the zero plane first, last, repeated, alone, under the three-term L_recon with
depth masks, and with an aperture (where the shortcut does not apply)."""
import numpy as np
import pytest

import oracle
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import rel_l2, to64, to_dev

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
LOSS_TOL = 1e-4

RGB = (638e-9, 520e-9, 450e-9)
CASES = {
    "zero-first-rgb": (inputs.custom(100, 120, 1500, wavelengths_m=RGB, z_m=(0.0, 5e-3, 10e-3),
                                     seed=41), 0.0, False),
    "zero-last": (inputs.custom(64, 96, 600, wavelengths_m=(520e-9, 450e-9), z_m=(3e-3, 0.0),
                                seed=42), 0.0, False),
    "zero-only": (inputs.custom(80, 80, 500, wavelengths_m=(638e-9,), z_m=(0.0,), seed=43),
                  0.0, False),
    "two-zero-planes": (inputs.custom(72, 100, 700, wavelengths_m=RGB, z_m=(0.0, 7e-3, 0.0),
                                      seed=44), 0.0, False),
    "zero-recon-masks": (inputs.custom(90, 120, 900, wavelengths_m=(638e-9, 450e-9),
                                       z_m=(0.0, 4e-3, 8e-3), seed=45), 0.0, True),
    "zero-with-aperture": (inputs.custom(64, 64, 400, wavelengths_m=(520e-9,),
                                         z_m=(0.0, 5e-3), seed=46), 40.0, False),
}


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


@pytest.mark.parametrize("identity", [1, 2])
@pytest.mark.parametrize("name", list(CASES))
def test_step_with_zero_planes_matches_oracle(name, identity, dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    w, aperture, recon = CASES[name]
    p = inputs.params_for(w)
    T = inputs.blob_targets(w.L, w.C, w.H, w.W, seed=47)
    M = inputs.depth_masks(w.L, w.H, w.W, seed=48) if recon else None
    plan = cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, aperture=aperture,
                    cutoff=w.cutoff, max_gaussians=w.N, device=dev,
                    tuning={"identity_planes": identity})
    assert plan.get_tuning()["identity_planes"] == identity
    Md = torch.from_numpy(M).to(dev) if recon else None
    if recon:
        plan.set_loss("recon", Md)
    pd, Td = to_dev(p, dev), torch.from_numpy(T).to(dev)
    loss, g = plan.step(pd, Td)
    fl = plan.forward_loss(pd, Td)
    ref = oracle.step(to64(p), T.astype(np.float64), w.H, w.W, w.wavelengths_m, w.pitch_m,
                      w.z_m, w.pad, w.cutoff, aperture=aperture, recon_mask=M,
                      loss="recon" if recon else "mse")
    assert abs(loss.item() - ref["loss"]) < LOSS_TOL * abs(ref["loss"])
    assert abs(fl.item() - ref["loss"]) < LOSS_TOL * abs(ref["loss"])
    for k in ref["grads"]:
        assert rel_l2(g[k].double().cpu().numpy(), ref["grads"][k]) < GRAD_TOL, k


def test_autograd_and_scaled_step_with_zero_planes(dev):
    """The autograd function (forward-only loss, then the recomputing fused step with the
    upstream gradient applied in the library) over a zero plane, against the oracle."""
    import torch
    from paper_2511_15022_gb300 import cgh
    from paper_2511_15022_gb300.autograd import hologram_loss
    w = CASES["zero-first-rgb"][0]
    p = inputs.params_for(w)
    T = inputs.blob_targets(w.L, w.C, w.H, w.W, seed=49)
    plan = cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, cutoff=w.cutoff,
                    max_gaussians=w.N, device=dev)
    leaves = {k: v.clone().requires_grad_(True) for k, v in to_dev(p, dev).items()}
    loss = hologram_loss(plan, leaves, torch.from_numpy(T).to(dev))
    (2.5 * loss).backward()
    ref = oracle.step(to64(p), T.astype(np.float64), w.H, w.W, w.wavelengths_m, w.pitch_m,
                      w.z_m, w.pad, w.cutoff)
    assert abs(loss.item() - ref["loss"]) < LOSS_TOL * abs(ref["loss"])
    for k in ref["grads"]:
        assert rel_l2(leaves[k].grad.double().cpu().numpy(), 2.5 * ref["grads"][k]) < GRAD_TOL, k


def test_identity_and_full_propagation_agree_at_1080p(dev):
    """The headline geometry (1080x1920, RGB, planes at 0 / 5 / 10 mm, 200k Gaussians) in the
    kernels the benchmark times: the fused step with the zero plane in the pixel domain
    against the same plan propagating every plane (identity_planes = 2)."""
    import torch
    from paper_2511_15022_gb300 import cgh
    w = inputs.hd_1080p()
    pd = to_dev(inputs.params_for(w), dev)
    Td = torch.from_numpy(inputs.blob_targets(w.L, w.C, w.H, w.W)).to(dev)
    plan = cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, cutoff=w.cutoff,
                    max_gaussians=w.N, device=dev)
    l1, g1 = plan.step(pd, Td)
    g1 = {k: v.clone() for k, v in g1.items()}
    plan.set_tuning(identity_planes=2)
    l2, g2 = plan.step(pd, Td)
    assert abs(l1.item() - l2.item()) < 1e-5 * abs(l2.item())
    for k in g1:
        assert rel_l2(g1[k].double().cpu().numpy(), g2[k].double().cpu().numpy()) < 1e-4, k
