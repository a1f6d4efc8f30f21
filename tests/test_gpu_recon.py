"""GPU parity of the reconstruction loss L_recon (Sec. 3.2) against the FP64 oracle: the
fused step, the forward-only loss and the pointwise loss entry point, with synthetic
binary depth masks, at the parity sizes of test_gpu_parity.py (tolerances as there)."""
import numpy as np
import pytest

import oracle
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import c64, rel_l2, to64, to_dev

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
LOSS_TOL = 1e-4
FIELD_TOL = 1e-4

CASES = {
    "small-256x256": inputs.small_256(),
    "odd-60x90-bandlimited": inputs.custom(60, 90, 300, wavelengths_m=(638e-9, 450e-9),
                                           z_m=(0.0, 50e-3), seed=11),
    "ragged-100x120-rgb": inputs.custom(100, 120, 1500, wavelengths_m=(638e-9, 520e-9, 450e-9),
                                        z_m=(0.0, 5e-3, 10e-3), seed=12),
}


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def make_plan(w, dev):
    from paper_2511_15022_gb300 import cgh
    return cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, pad=w.pad, cutoff=w.cutoff,
                    max_gaussians=max(w.N, 1), device=dev)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("with_mask", [True, False])
def test_step_recon_matches_oracle(name, with_mask, dev):
    import torch
    w = CASES[name]
    p = inputs.params_for(w)
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    M = inputs.depth_masks(w.L, w.H, w.W, seed=31) if with_mask else None
    plan = make_plan(w, dev)
    plan.set_loss("recon", torch.from_numpy(M).to(dev) if with_mask else None)
    pd, Td = to_dev(p, dev), torch.from_numpy(T).to(dev)
    loss, g = plan.step(pd, Td)
    ref = oracle.step(to64(p), T.astype(np.float64), w.H, w.W, w.wavelengths_m, w.pitch_m,
                      w.z_m, w.pad, w.cutoff, recon_mask=M, loss="recon")
    assert abs(loss.item() - ref["loss"]) < LOSS_TOL * abs(ref["loss"])
    for k in ref["grads"]:
        assert rel_l2(g[k].double().cpu().numpy(), ref["grads"][k]) < GRAD_TOL, k
    fl = plan.forward_loss(pd, Td)
    assert abs(fl.item() - loss.item()) <= 1e-6 * abs(loss.item())
    # back to the plain intensity loss
    plan.set_loss("mse")
    ref_mse = oracle.step(to64(p), T.astype(np.float64), w.H, w.W, w.wavelengths_m, w.pitch_m,
                          w.z_m, w.pad, w.cutoff)
    assert abs(plan.forward_loss(pd, Td).item() - ref_mse["loss"]) < LOSS_TOL * ref_mse["loss"]


def test_intensity_loss_recon(dev):
    import torch
    w = CASES["ragged-100x120-rgb"]
    plan = make_plan(w, dev)
    M = inputs.depth_masks(w.L, w.H, w.W, seed=32)
    plan.set_loss("recon", torch.from_numpy(M).to(dev))
    Ud = np.stack([inputs.random_field(w.C, w.H, w.W, seed=60 + l) for l in range(w.L)]) * 0.5
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    loss, dUd = plan.intensity_loss(torch.from_numpy(Ud).to(dev), torch.from_numpy(T).to(dev))
    rl, rd = oracle.recon_loss(Ud.astype(np.complex128), T.astype(np.float64), M)
    assert abs(loss.item() - rl) < LOSS_TOL * rl
    assert rel_l2(c64(dUd), rd) < FIELD_TOL


def test_set_loss_rejects_a_mask_without_recon(dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    w = CASES["small-256x256"]
    plan = make_plan(w, dev)
    M = torch.zeros((w.L, w.H, w.W), dtype=torch.uint8, device=dev)
    lib = cgh.load()
    import ctypes
    st = lib.cgh_plan_set_loss(plan._h, 0, ctypes.c_void_p(M.data_ptr()))
    assert st == 1
    with pytest.raises(KeyError):
        plan.set_loss("ssim")
