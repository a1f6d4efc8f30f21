"""The torch.autograd.Function (forward recomputed in the backward pass, Sec. 3.4) on the
GPU: loss and parameter gradients against the FP64 oracle, the upstream gradient applied
inside the library, reuse of the forward's binning only while it is still the caller's, the
eager form (gradients computed in the forward, no recompute) against the recomputing one,
and the gradients of a 64x64 crop of the 1080p RGB three-plane workload against central
differences of the oracle's forward loss."""
import numpy as np
import pytest

import oracle
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import rel_l2, to64, to_dev

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
LOSS_TOL = 1e-4

RGB = (638e-9, 520e-9, 450e-9)
PLANES = (0.0, 5e-3, 10e-3)


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


def leaf_params(p, dev):
    return {k: v.clone().requires_grad_(True) for k, v in to_dev(p, dev).items()}


def autograd_grads(plan, params, target, scale=1.0):
    from paper_2511_15022_gb300.autograd import hologram_loss
    loss = hologram_loss(plan, params, target)
    (loss * scale if scale != 1.0 else loss).backward()
    return loss.item(), {k: v.grad.detach().clone() for k, v in params.items()}


def test_autograd_matches_oracle(dev):
    import torch
    w = inputs.custom(100, 120, 1500, wavelengths_m=RGB, z_m=PLANES, seed=12)
    p = inputs.params_for(w)
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    plan = make_plan(w, dev)
    loss, g = autograd_grads(plan, leaf_params(p, dev), torch.from_numpy(T).to(dev))
    ref = oracle.step(to64(p), T.astype(np.float64), w.H, w.W, w.wavelengths_m, w.pitch_m,
                      w.z_m, w.pad, w.cutoff)
    assert abs(loss - ref["loss"]) < LOSS_TOL * abs(ref["loss"])
    for k in ref["grads"]:
        assert rel_l2(g[k].double().cpu().numpy(), ref["grads"][k]) < GRAD_TOL, k


def test_upstream_gradient_scales_every_gradient(dev):
    """(s L).backward() hands s to the library, which applies it to the raster moments."""
    import torch
    w = inputs.custom(60, 90, 400, wavelengths_m=RGB[:2], z_m=(0.0, 4e-3), seed=31)
    p = inputs.params_for(w)
    T = torch.from_numpy(inputs.blob_targets(w.L, w.C, w.H, w.W)).to(dev)
    plan = make_plan(w, dev)
    _, g1 = autograd_grads(plan, leaf_params(p, dev), T)
    _, g3 = autograd_grads(plan, leaf_params(p, dev), T, scale=-2.5)
    for k in g1:
        assert rel_l2(g3[k].double().cpu().numpy(), -2.5 * g1[k].double().cpu().numpy()) < 1e-5, k


def test_eager_mode_equals_recompute(dev):
    """hologram_loss(..., eager=True) runs the fused forward and backward inside the autograd
    forward and keeps only the O(N) parameter gradients, which backward multiplies by the
    upstream scalar: the same loss and gradients as the recomputing path, scaled alike."""
    import torch
    from paper_2511_15022_gb300.autograd import hologram_loss
    w = inputs.custom(80, 100, 900, wavelengths_m=RGB, z_m=PLANES, seed=41)
    p = inputs.params_for(w)
    T = torch.from_numpy(inputs.blob_targets(w.L, w.C, w.H, w.W)).to(dev)
    plan = make_plan(w, dev)

    def run(eager, scale):
        params = leaf_params(p, dev)
        loss = hologram_loss(plan, params, T, eager=eager)
        (loss * scale).backward()
        return loss.item(), {k: v.grad.double().cpu().numpy() for k, v in params.items()}

    l0, g0 = run(False, 1.0)
    l1, g1 = run(True, 1.0)
    _, g2 = run(True, -2.5)
    assert abs(l1 - l0) < 1e-5 * abs(l0)
    for k in g0:
        assert rel_l2(g1[k], g0[k]) < 1e-5, k
        # separate steps: the raster backward's atomics add in a different order each run
        assert rel_l2(g2[k], -2.5 * g1[k]) < 1e-5, k


def test_binning_reuse_equals_rebinning(dev):
    """cgh_step_scaled with reuse_binning after a forward on the same parameters gives what
    a full rebinning gives (only the order of equal-tile Gaussians may differ)."""
    import torch
    w = inputs.custom(100, 120, 1500, wavelengths_m=RGB, z_m=PLANES, seed=33)
    p = to_dev(inputs.params_for(w), dev)
    T = torch.from_numpy(inputs.blob_targets(w.L, w.C, w.H, w.W)).to(dev)
    plan = make_plan(w, dev)
    l0, g0 = plan.step(p, T)
    plan.forward_loss(p, T)
    l1, g1 = plan.step(p, T, reuse_binning=True)
    assert abs(l1.item() - l0.item()) <= 1e-5 * abs(l0.item())
    for k in g0:
        assert rel_l2(g1[k].double().cpu().numpy(), g0[k].double().cpu().numpy()) < 1e-5, k


def test_intervening_call_forces_rebinning(dev):
    """A call on the plan between forward and backward rebins other parameters in the
    workspace: the backward must notice and rebin its own."""
    import torch
    w = inputs.custom(80, 96, 900, wavelengths_m=RGB, z_m=PLANES, seed=34)
    pa = inputs.params_for(w)
    pb = inputs.params_for(w, seed=35)
    T = torch.from_numpy(inputs.blob_targets(w.L, w.C, w.H, w.W)).to(dev)
    plan = make_plan(w, dev)
    _, ref = plan.step(to_dev(pa, dev), T)
    from paper_2511_15022_gb300.autograd import hologram_loss
    params = leaf_params(pa, dev)
    loss = hologram_loss(plan, params, T)
    plan.forward_loss(to_dev(pb, dev), T)  # same shapes, other values and pointers
    loss.backward()
    for k in ref:
        assert rel_l2(params[k].grad.double().cpu().numpy(), ref[k].double().cpu().numpy()) < 1e-5, k


def test_in_place_change_before_backward_is_rejected(dev):
    """The saved parameters share the callers' version counters: changing a parameter in
    place between forward and backward (which would also make the reused binning stale)
    is an autograd error, not a silently wrong gradient."""
    import torch
    w = inputs.custom(40, 60, 200, seed=36)
    T = torch.from_numpy(inputs.blob_targets(w.L, w.C, w.H, w.W)).to(dev)
    plan = make_plan(w, dev)
    from paper_2511_15022_gb300.autograd import hologram_loss
    params = leaf_params(inputs.params_for(w), dev)
    loss = hologram_loss(plan, params, T)
    with torch.no_grad():
        params["theta"].add_(0.25)
    with pytest.raises(RuntimeError):
        loss.backward()


def test_gradients_against_finite_differences_on_a_64x64_crop(dev):
    """A 64x64 window of the 1080p workload (RGB, planes 0/5/10 mm, its Gaussian density:
    200k / (1080 * 1920) per pixel, its scale and opacity distributions): every parameter
    kind's autograd gradient against central differences of the FP64 oracle's loss."""
    import torch
    N = round(200_000 * 64 * 64 / (1080 * 1920))
    w = inputs.custom(64, 64, N, wavelengths_m=RGB, z_m=PLANES, seed=37)
    p = inputs.params_for(w)
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    plan = make_plan(w, dev)
    _, g = autograd_grads(plan, leaf_params(p, dev), torch.from_numpy(T).to(dev))
    q0 = to64(p)
    T64 = T.astype(np.float64)

    def loss(q):
        _, Ud = oracle.forward(q, w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, w.pad, w.cutoff)
        return oracle.mse_loss(Ud, T64)[0]

    rng = np.random.default_rng(38)
    for key in q0:
        gk = g[key].double().cpu().numpy()
        floor = 2e-3 * np.sqrt(np.mean(gk ** 2))
        # the Gaussians with the largest gradients of this kind, and two random ones
        flat = np.argsort(-np.abs(gk).reshape(-1))[:2].tolist() + \
            rng.choice(gk.size, 2, replace=False).tolist()
        for f in flat:
            idx = np.unravel_index(f, gk.shape)
            h = 1e-6 * max(1.0, abs(q0[key][idx]))
            qp = {k: v.copy() for k, v in q0.items()}
            qm = {k: v.copy() for k, v in q0.items()}
            qp[key][idx] += h
            qm[key][idx] -= h
            fd = (loss(qp) - loss(qm)) / (2 * h)
            assert abs(gk[idx] - fd) <= 2e-3 * abs(fd) + floor, (key, idx, gk[idx], fd)


def test_step_scaled_argument_checks(dev):
    """The upstream scale must be one float32 element on the plan's device."""
    import torch
    w = inputs.custom(32, 48, 50, seed=48)
    p = to_dev(inputs.params_for(w), dev)
    T = torch.from_numpy(inputs.blob_targets(w.L, w.C, w.H, w.W)).to(dev)
    plan = make_plan(w, dev)
    for bad in (torch.ones(1, dtype=torch.float64, device=dev), torch.ones(2, device=dev),
                torch.ones(1)):
        with pytest.raises(ValueError):
            plan.step(p, T, grad_scale=bad)
    _, g0 = plan.step(p, T)
    # the same binning for both calls: the tile lists' order comes from atomic cursors, so a
    # rebinned call sums each pixel's Gaussians in another FP32 order
    _, g2 = plan.step(p, T, grad_scale=torch.full((1,), 2.0, device=dev), reuse_binning=True)
    for k in g0:
        assert rel_l2(g2[k].double().cpu().numpy(), 2.0 * g0[k].double().cpu().numpy()) < 1e-5, k


def test_hologram_intensity_matches_oracle(dev):
    """HologramIntensity: the intensities I_l = |U(d_l)|^2 (Sec. 3.2) against the oracle's
    forward, and the gradients of a weighted sum of them, sum(w I), against the oracle's
    chain dL/dUd = 2 w Ud -> adjoint propagation -> raster backward."""
    import torch
    from paper_2511_15022_gb300.autograd import hologram_intensity
    w = inputs.custom(96, 128, 1200, wavelengths_m=RGB, z_m=PLANES, seed=14)
    p = inputs.params_for(w)
    plan = make_plan(w, dev)
    params = leaf_params(p, dev)
    I = hologram_intensity(plan, params)
    wt = np.random.default_rng(15).uniform(-1.0, 1.0, size=I.shape).astype(np.float32)
    (I * torch.from_numpy(wt).to(dev)).sum().backward()
    U0, Ud = oracle.forward(to64(p), w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, w.pad, w.cutoff)
    assert rel_l2(I.detach().double().cpu().numpy(), np.abs(Ud) ** 2) < LOSS_TOL
    dU0 = oracle.blasm_bwd(2.0 * wt.astype(np.float64) * Ud, w.wavelengths_m, w.pitch_m, w.z_m, w.pad)
    ref = oracle.raster_bwd(to64(p), w.H, w.W, dU0, w.cutoff)
    for k in ref:
        assert rel_l2(params[k].grad.double().cpu().numpy(), ref[k]) < GRAD_TOL, k
