"""Parity at the full 1080x1920, RGB, three-plane, 200k-Gaussian workload in the launch
configuration the benchmark times: sampled outputs the oracle computes one by one
(pixels of the field, Gaussians of the gradient, one channel of the propagation), and
whole-tensor properties (fused step == composition of the verified entry points)."""
import numpy as np
import pytest

import oracle
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import c64, rel_l2, to64, to_dev

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-4
GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15022_gb300 import cgh
    dev = torch.device("cuda", 0)
    w = inputs.hd_1080p()
    p = inputs.params_for(w)
    plan = cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, cutoff=w.cutoff,
                    max_gaussians=w.N, device=dev)
    return w, p, plan, dev


def test_raster_fwd_sampled_pixels(setup):
    w, p, plan, dev = setup
    U = plan.raster_fwd(to_dev(p, dev))
    idx = inputs.sample_indices(1500, w.H * w.W, seed=61)
    # include the four corners and the last row/column
    idx = np.unique(np.concatenate([idx, [0, w.W - 1, (w.H - 1) * w.W, w.H * w.W - 1]]))
    got = c64(U).reshape(w.C, -1)[:, idx]
    ref = oracle.raster_fwd(to64(p), w.H, w.W, w.cutoff, pix_idx=idx)
    assert rel_l2(got, ref) < FIELD_TOL


def test_raster_bwd_sampled_gaussians(setup):
    import torch
    w, p, plan, dev = setup
    dU = inputs.random_field(w.C, w.H, w.W, seed=62)
    g = plan.raster_bwd(to_dev(p, dev), torch.from_numpy(dU).to(dev))
    sel = inputs.sample_indices(24, w.N, seed=63)
    ref = oracle.raster_bwd(to64(p), w.H, w.W, dU, w.cutoff, g_idx=sel)
    for k in ref:
        assert rel_l2(g[k].double().cpu().numpy()[sel], ref[k]) < GRAD_TOL, k


def test_blasm_fwd_one_channel_plane(setup):
    """Full-size propagation: the 450 nm channel at 10 mm against the oracle."""
    import torch
    w, p, plan, dev = setup
    U0 = inputs.random_field(w.C, w.H, w.W, seed=64)
    Ud = plan.blasm_fwd(torch.from_numpy(U0).to(dev))
    c, l = 2, 2
    ref = oracle.blasm_fwd(U0[c:c + 1], [w.wavelengths_m[c]], w.pitch_m, [w.z_m[l]], w.pad)
    assert rel_l2(c64(Ud[l, c]), ref[0, 0]) < FIELD_TOL


def test_fused_step_equals_composition(setup):
    """cgh_step == raster_fwd -> blasm_fwd -> intensity_loss -> blasm_bwd -> raster_bwd,
    each of which is checked against the oracle above or at smaller sizes."""
    import torch
    w, p, plan, dev = setup
    T = torch.from_numpy(inputs.blob_targets(w.L, w.C, w.H, w.W)).to(dev)
    pd = to_dev(p, dev)
    loss, g = plan.step(pd, T)
    U0 = plan.raster_fwd(pd)
    Ud = plan.blasm_fwd(U0)
    l2, dUd = plan.intensity_loss(Ud, T)
    dU0 = plan.blasm_bwd(dUd)
    g2 = plan.raster_bwd(pd, dU0)
    assert abs(loss.item() - l2.item()) < 1e-5 * l2.item()
    for k in g:
        assert rel_l2(g[k].double().cpu().numpy(), g2[k].double().cpu().numpy()) < 1e-4, k
    st = plan.status()
    assert not st["overflow"] and not st["nonfinite"]


def test_blasm_fwd_one_channel_all_planes(setup):
    """Full-size propagation of the 638 nm channel to all three planes (0, 5 and 10 mm) in
    the kernels the benchmark times, against the oracle."""
    import torch
    w, p, plan, dev = setup
    U0 = inputs.random_field(w.C, w.H, w.W, seed=66)
    Ud = plan.blasm_fwd(torch.from_numpy(U0).to(dev))
    c = 0
    ref = oracle.blasm_fwd(U0[c:c + 1], [w.wavelengths_m[c]], w.pitch_m, list(w.z_m), w.pad)
    for l in range(w.L):
        assert rel_l2(c64(Ud[l, c]), ref[l, 0]) < FIELD_TOL, l


def test_blasm_bwd_one_channel_all_planes(setup):
    """Adjoint propagation (Suppl. BLASM backward: conj(H) under the same band limit, summed
    over the planes) at full size in the kernels the benchmark times: dL/dUd non-zero in one
    channel only, so the oracle needs only that channel; the other channels must stay zero."""
    import torch
    w, p, plan, dev = setup
    c = 1
    dUd = np.zeros((w.L, w.C, w.H, w.W), np.complex64)
    dUd[:, c] = inputs.random_field(w.L, w.H, w.W, seed=65)
    dU0 = c64(plan.blasm_bwd(torch.from_numpy(dUd).to(dev)))
    ref = oracle.blasm_bwd(dUd[:, c:c + 1], [w.wavelengths_m[c]], w.pitch_m, list(w.z_m), w.pad)
    assert rel_l2(dU0[c], ref[0]) < FIELD_TOL
    for other in range(w.C):
        if other != c:
            assert np.abs(dU0[other]).max() == 0.0, other
