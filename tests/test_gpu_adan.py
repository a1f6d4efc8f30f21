"""GPU Adan (cgh_adan_step) and the aperture option against the FP64 oracle.

Adan: five steps on three groups with seeded FP32 gradients; the parameter changes agree
with the oracle's to 1e-5 (relative L2; FP32 rounding of each update).
Aperture: the fused step with the index-space aperture of Algorithm 3 switched on, at the
parity tolerances of test_gpu_parity.py (field 1e-4, gradients 1e-3, loss 1e-4)."""
import numpy as np
import pytest

import oracle
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import rel_l2, to64, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def test_adan_matches_oracle(dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    rng = np.random.default_rng(5)
    sizes, lrs = (1000, 37, 4097), (1e-2, 5e-3, 2.5e-2)
    p0 = [rng.standard_normal(n).astype(np.float32) for n in sizes]
    grads = [[rng.standard_normal(n).astype(np.float32) for n in sizes] for _ in range(5)]
    P = [torch.from_numpy(a).to(dev) for a in p0]
    state = [[torch.zeros_like(a) for _ in range(4)] for a in P]
    ref = [a.astype(np.float64) for a in p0]
    rstate = [[np.zeros(n) for _ in range(4)] for n in sizes]
    for t, gs in enumerate(grads, start=1):
        G = [torch.from_numpy(g).to(dev) for g in gs]
        cgh.adan_step([(P[i], G[i], *state[i], lrs[i]) for i in range(3)], t)
        for i in range(3):
            oracle.adan(ref[i], gs[i].astype(np.float64), *rstate[i], lrs[i], t)
    for i in range(3):
        got = P[i].cpu().numpy().astype(np.float64)
        assert rel_l2(got - p0[i], ref[i] - p0[i]) < 1e-5, i


def test_step_with_aperture_matches_oracle(dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    w = inputs.custom(100, 120, 1500, wavelengths_m=(638e-9, 520e-9, 450e-9),
                      z_m=(0.0, 5e-3, 10e-3), seed=12)
    aperture = 60.0
    p = inputs.params_for(w)
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    plan = cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, pad=w.pad, aperture=aperture,
                    cutoff=w.cutoff, max_gaussians=w.N, device=dev)
    loss, g = plan.step(to_dev(p, dev), torch.from_numpy(T).to(dev))
    ref = oracle.step(to64(p), T.astype(np.float64), w.H, w.W, w.wavelengths_m, w.pitch_m,
                      w.z_m, w.pad, w.cutoff, aperture)
    assert abs(loss.item() - ref["loss"]) < 1e-4 * ref["loss"]
    for k in ref["grads"]:
        assert rel_l2(g[k].double().cpu().numpy(), ref["grads"][k]) < 1e-3, k
    # the aperture removes energy: the propagated field differs from the unfiltered one
    plan0 = cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, pad=w.pad, cutoff=w.cutoff,
                     max_gaussians=w.N, device=dev)
    assert abs(plan0.forward_loss(to_dev(p, dev), torch.from_numpy(T).to(dev)).item() - loss.item()) > 1e-6
