"""GPU parity of the POH conversion (Sec. 3.3) against the FP64 oracle: the smooth POH
(DPAC) and the random POH field elementwise, and the joint conversion step (loss, Gaussian
gradients, phase gradient) with and without depth masks.  Tolerances as in
test_gpu_parity.py: fields 1e-4, gradients 1e-3, loss 1e-4 (relative)."""
import numpy as np
import pytest

import oracle
from oracle import poh_ref as pr
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import c64, rel_l2, to64, to_dev

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-4
GRAD_TOL = 1e-3
LOSS_TOL = 1e-4

CASES = {
    "small-256x256": inputs.small_256(),
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


def test_dpac_and_field(dev):
    import torch
    w = CASES["ragged-100x120-rgb"]
    plan = make_plan(w, dev)
    U = inputs.random_field(w.C, w.H, w.W, seed=70) * 0.7
    for mode in ("double", "printed"):
        got = c64(plan.poh_dpac(torch.from_numpy(U).to(dev), mode=mode))
        assert rel_l2(got, pr.dpac(U.astype(np.complex128), mode=mode)) < FIELD_TOL, mode
    rng = np.random.default_rng(71)
    phi = rng.uniform(-np.pi, np.pi, size=(w.C, w.H, w.W)).astype(np.float32)
    got = c64(plan.poh_field(torch.from_numpy(phi).to(dev)))
    assert rel_l2(got, pr.poh_field(phi.astype(np.float64))) < FIELD_TOL


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("with_mask", [True, False])
def test_poh_step_matches_oracle(name, with_mask, dev):
    import torch
    w = CASES[name]
    p = inputs.params_for(w)
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    M = inputs.depth_masks(w.L, w.H, w.W, seed=33) if with_mask else None
    rng = np.random.default_rng(72)
    phi = rng.uniform(-np.pi, np.pi, size=(w.C, w.H, w.W)).astype(np.float32)
    plan = make_plan(w, dev)
    if with_mask:
        plan.set_loss("recon", torch.from_numpy(M).to(dev))
    loss, g, dphi = plan.poh_step(to_dev(p, dev), torch.from_numpy(phi).to(dev),
                                  torch.from_numpy(T).to(dev), 0.1, 0.01)
    ref = pr.poh_step(to64(p), phi.astype(np.float64), T.astype(np.float64), w.H, w.W,
                      w.wavelengths_m, w.pitch_m, w.z_m, w.pad, w.cutoff, M, 0.1, 0.01)
    assert abs(loss.item() - ref["loss"]) < LOSS_TOL * abs(ref["loss"])
    for k in ref["grads"]:
        assert rel_l2(g[k].double().cpu().numpy(), ref["grads"][k]) < GRAD_TOL, k
    assert rel_l2(dphi.double().cpu().numpy(), ref["dphi"]) < GRAD_TOL
