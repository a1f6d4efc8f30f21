"""GPU parity of the C-ABI path against the FP64 oracle.

Tolerances (relative L2 over the whole compared tensor): complex fields 1e-4, gradients
1e-3 per parameter kind, loss 1e-4.  Sizes span several 16x16 tiles with ragged edges,
odd image sizes, band-limited and unmasked propagation, smooth mode, the 0.99 cap, and
empty / off-screen / single-row inputs.  Every call goes through libcgh's C ABI.
"""
import numpy as np
import pytest

import oracle
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import c64, rel_l2, to64, to_dev

FIELD_TOL = 1e-4
GRAD_TOL = 1e-3
LOSS_TOL = 1e-4

pytestmark = pytest.mark.gpu

CASES = {
    "small-256x256": inputs.small_256(),
    "odd-60x90-bandlimited": inputs.custom(60, 90, 300, wavelengths_m=(638e-9, 450e-9),
                                           z_m=(0.0, 50e-3), seed=11),
    "ragged-100x120-rgb": inputs.custom(100, 120, 1500, wavelengths_m=(638e-9, 520e-9, 450e-9),
                                        z_m=(0.0, 5e-3, 10e-3), seed=12),
    "single-row-1x64": inputs.custom(1, 64, 40, z_m=(2e-3,), seed=13),
}


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def make_plan(w, dev, **kw):
    from paper_2511_15022_gb300 import cgh
    return cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, pad=w.pad,
                    cutoff=kw.pop("cutoff", w.cutoff), max_gaussians=max(w.N, 1), device=dev, **kw)


@pytest.mark.parametrize("name", list(CASES))
def test_raster_fwd(name, dev):
    w = CASES[name]
    p = inputs.params_for(w)
    plan = make_plan(w, dev)
    U = c64(plan.raster_fwd(to_dev(p, dev)))
    ref = oracle.raster_fwd(to64(p), w.H, w.W, w.cutoff)
    assert rel_l2(U, ref) < FIELD_TOL


def test_raster_with_gaussians_spanning_hundreds_of_tiles(dev):
    """Scales up to 40 px (boxes of up to ~16 x 16 tiles, the size optimised Gaussians grow
    to): the tile emit deals each warp's pooled (Gaussian, tile) items to its lanes; field
    and sampled gradients against the oracle."""
    import torch
    w = inputs.custom(384, 512, 700, s_min_px=0.5, s_max_px=40.0, seed=45)
    p = inputs.params_for(w)
    plan = make_plan(w, dev)
    U = c64(plan.raster_fwd(to_dev(p, dev)))
    ref = oracle.raster_fwd(to64(p), w.H, w.W, w.cutoff)
    assert rel_l2(U, ref) < FIELD_TOL
    dU = inputs.random_field(w.C, w.H, w.W, seed=46)
    g = plan.raster_bwd(to_dev(p, dev), torch.from_numpy(dU).to(dev))
    sel = inputs.sample_indices(24, w.N, seed=47)
    gref = oracle.raster_bwd(to64(p), w.H, w.W, dU, w.cutoff, g_idx=sel)
    for k in gref:
        assert rel_l2(g[k].double().cpu().numpy()[sel], gref[k]) < GRAD_TOL, k
    assert plan.status()["pairs"] > 8 * w.N  # many tiles per Gaussian on average


def test_raster_with_more_tiles_than_one_scan_chunk(dev):
    """2304 x 4096 pixels = 36,864 tiles: the tile scan runs in two chunks joined by a
    carry; the field on sampled pixels (all of the first and last tile rows included) and
    the gradients of sampled Gaussians against the oracle."""
    import torch
    w = inputs.custom(2304, 4096, 6000, seed=41)
    p = inputs.params_for(w)
    plan = make_plan(w, dev)
    U = c64(plan.raster_fwd(to_dev(p, dev))).reshape(w.C, -1)
    rows = np.concatenate([np.arange(0, 16), np.arange(w.H - 16, w.H)])
    edge = (rows[:, None] * w.W + np.arange(0, w.W, 7)[None, :]).reshape(-1)
    idx = np.unique(np.concatenate([inputs.sample_indices(3000, w.H * w.W, seed=42), edge]))
    ref = oracle.raster_fwd(to64(p), w.H, w.W, w.cutoff, pix_idx=idx)
    assert rel_l2(U[:, idx], ref) < FIELD_TOL
    dU = inputs.random_field(w.C, w.H, w.W, seed=43)
    g = plan.raster_bwd(to_dev(p, dev), torch.from_numpy(dU).to(dev))
    sel = inputs.sample_indices(16, w.N, seed=44)
    gref = oracle.raster_bwd(to64(p), w.H, w.W, dU, w.cutoff, g_idx=sel)
    for k in gref:
        assert rel_l2(g[k].double().cpu().numpy()[sel], gref[k]) < GRAD_TOL, k


@pytest.mark.parametrize("name", list(CASES))
def test_blasm_fwd_bwd(name, dev):
    import torch
    w = CASES[name]
    plan = make_plan(w, dev)
    U0 = inputs.random_field(w.C, w.H, w.W, seed=21)
    Ud = c64(plan.blasm_fwd(torch.from_numpy(U0).to(dev)))
    ref = oracle.blasm_fwd(U0, w.wavelengths_m, w.pitch_m, w.z_m, w.pad)
    assert rel_l2(Ud, ref) < FIELD_TOL
    dUd = np.stack([inputs.random_field(w.C, w.H, w.W, seed=30 + l) for l in range(w.L)])
    dU0 = c64(plan.blasm_bwd(torch.from_numpy(dUd).to(dev)))
    ref = oracle.blasm_bwd(dUd, w.wavelengths_m, w.pitch_m, w.z_m, w.pad)
    assert rel_l2(dU0, ref) < FIELD_TOL


@pytest.mark.parametrize("name", list(CASES))
def test_raster_bwd(name, dev):
    import torch
    w = CASES[name]
    p = inputs.params_for(w)
    plan = make_plan(w, dev)
    dU = inputs.random_field(w.C, w.H, w.W, seed=41)
    g = plan.raster_bwd(to_dev(p, dev), torch.from_numpy(dU).to(dev))
    ref = oracle.raster_bwd(to64(p), w.H, w.W, dU, w.cutoff)
    for k in ref:
        assert rel_l2(g[k].double().cpu().numpy(), ref[k]) < GRAD_TOL, k


@pytest.mark.parametrize("name", list(CASES))
def test_step_matches_oracle(name, dev):
    import torch
    w = CASES[name]
    p = inputs.params_for(w)
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    plan = make_plan(w, dev)
    pd, Td = to_dev(p, dev), torch.from_numpy(T).to(dev)
    loss, g = plan.step(pd, Td)
    ref = oracle.step(to64(p), T.astype(np.float64), w.H, w.W, w.wavelengths_m, w.pitch_m,
                      w.z_m, w.pad, w.cutoff)
    assert abs(loss.item() - ref["loss"]) < LOSS_TOL * abs(ref["loss"])
    for k in ref["grads"]:
        assert rel_l2(g[k].double().cpu().numpy(), ref["grads"][k]) < GRAD_TOL, k
    # forward-only entry point gives the same loss
    fl = plan.forward_loss(pd, Td)
    assert abs(fl.item() - loss.item()) <= 1e-6 * abs(loss.item())


def test_intensity_loss(dev):
    import torch
    w = CASES["ragged-100x120-rgb"]
    plan = make_plan(w, dev)
    Ud = np.stack([inputs.random_field(w.C, w.H, w.W, seed=50 + l) for l in range(w.L)]) * 0.5
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    loss, dUd = plan.intensity_loss(torch.from_numpy(Ud).to(dev), torch.from_numpy(T).to(dev))
    rl, rd = oracle.mse_loss(Ud.astype(np.complex128), T.astype(np.float64))
    assert abs(loss.item() - rl) < LOSS_TOL * rl
    assert rel_l2(c64(dUd), rd) < FIELD_TOL


def test_band_limits_bit_exact(dev):
    """The integer band-limit decisions equal the oracle's mask bit for bit."""
    w = CASES["odd-60x90-bandlimited"]
    plan = make_plan(w, dev)
    kx, ky = plan.band_limits()
    for c, lam in enumerate(w.wavelengths_m):
        for l, z in enumerate(w.z_m):
            Hf = oracle.blasm_transfer(2 * w.H, 2 * w.W, lam, w.pitch_m, z)
            mask = np.abs(Hf) > 0
            sx = np.fft.fftfreq(2 * w.W, d=1.0 / (2 * w.W)).astype(int)
            sy = np.fft.fftfreq(2 * w.H, d=1.0 / (2 * w.H)).astype(int)
            mine = (np.abs(sx)[None, :] <= kx[c * w.L + l]) & (np.abs(sy)[:, None] <= ky[c * w.L + l])
            assert np.array_equal(mine, mask)
    # the 50 mm plane is band-limited on this grid, the 0 mm one is not
    assert kx[1] < w.W and kx[0] == w.W


def test_smooth_mode_and_alpha_cap(dev):
    """cutoff = 0 (every pair kept, power clamp -50) and opacities near 1 (0.99 cap)."""
    import torch
    w = inputs.custom(40, 48, 120, wavelengths_m=(520e-9, 450e-9), z_m=(3e-3,), seed=14,
                      cutoff=0.0)
    p = inputs.params_for(w)
    p["alpha_raw"][::2] = 6.0  # alpha = 0.9975: the cap binds near the mean
    plan = make_plan(w, dev)
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    loss, g = plan.step(to_dev(p, dev), torch.from_numpy(T).to(dev))
    ref = oracle.step(to64(p), T.astype(np.float64), w.H, w.W, w.wavelengths_m, w.pitch_m,
                      w.z_m, w.pad, cutoff=0.0)
    assert abs(loss.item() - ref["loss"]) < LOSS_TOL * abs(ref["loss"])
    for k in ref["grads"]:
        assert rel_l2(g[k].double().cpu().numpy(), ref["grads"][k]) < GRAD_TOL, k


def test_empty_and_offscreen(dev):
    import torch
    w = inputs.custom(32, 48, 8, seed=15)
    plan = make_plan(w, dev)
    # N = 0: zero field, zero-size gradients
    p0 = {k: v[:0] for k, v in inputs.params_for(w).items()}
    U = plan.raster_fwd(to_dev(p0, dev))
    assert float(U.abs().max()) == 0.0
    # Gaussians pushed to the image corner (x -> W, y -> 0): mostly clipped by the edge
    p = inputs.params_for(w)
    p["xy_raw"][:, 0] = 8.0
    p["xy_raw"][:, 1] = -8.0
    p["s_raw"][:] = np.log(0.5)
    U = c64(plan.raster_fwd(to_dev(p, dev)))
    ref = oracle.raster_fwd(to64(p), w.H, w.W, w.cutoff)
    assert np.abs(U - ref).max() < 1e-6
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    loss, g = plan.step(to_dev(p, dev), torch.from_numpy(T).to(dev))
    refs = oracle.step(to64(p), T.astype(np.float64), w.H, w.W, w.wavelengths_m, w.pitch_m,
                       w.z_m, w.pad, w.cutoff)
    for k in refs["grads"]:
        assert np.abs(g[k].double().cpu().numpy() - refs["grads"][k]).max() < 1e-6


def test_capacity_overflow_is_exact(dev):
    """A list capacity far below the pair count routes tiles through the exhaustive path:
    same field, overflow flagged."""
    w = CASES["ragged-100x120-rgb"]
    p = inputs.params_for(w)
    plan = make_plan(w, dev, tuning={"pair_capacity_per_gaussian": 1})
    U = c64(plan.raster_fwd(to_dev(p, dev)))
    st = plan.status()
    assert st["overflow"] and st["pairs"] > w.N
    ref = oracle.raster_fwd(to64(p), w.H, w.W, w.cutoff)
    assert rel_l2(U, ref) < FIELD_TOL


def test_nonfinite_parameters_are_flagged_and_skipped(dev):
    w = inputs.custom(32, 32, 50, seed=16)
    p = inputs.params_for(w)
    p["theta"][3] = np.nan
    plan = make_plan(w, dev)
    U = c64(plan.raster_fwd(to_dev(p, dev)))
    assert plan.status()["nonfinite"]
    q = {k: np.delete(v, 3, axis=0) for k, v in p.items()}
    ref = oracle.raster_fwd(to64(q), w.H, w.W, w.cutoff)
    assert rel_l2(U, ref) < FIELD_TOL


@pytest.mark.parametrize("case,tuning", [
    ("ragged-100x120-rgb", {"col_block": 1, "row_block": 1}),
    ("ragged-100x120-rgb", {"col_block": 2, "row_block": 3, "fft_threads": 128}),
    ("small-256x256", {"fft_kernels": 2}),
])
def test_tuning_variants_agree(case, tuning, dev):
    """Other block shapes, and the generic FFT kernels instead of the specialised ones,
    give the same step."""
    import torch
    w = CASES[case]
    p = inputs.params_for(w)
    T = inputs.blob_targets(w.L, w.C, w.H, w.W)
    pd, Td = to_dev(p, dev), torch.from_numpy(T).to(dev)
    base_loss, base_g = make_plan(w, dev).step(pd, Td)
    loss, g = make_plan(w, dev, tuning=tuning).step(pd, Td)
    assert abs(loss.item() - base_loss.item()) < 1e-5 * base_loss.item()
    for k in g:
        assert rel_l2(g[k].cpu().numpy(), base_g[k].cpu().numpy()) < 1e-4
