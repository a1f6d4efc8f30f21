"""Work counters of the rasteriser sweeps (cgh_raster_stats) through the C ABI.

The contributing-pair count is checked against a brute-force FP64 count over every
(pixel, Gaussian) pair built on the oracle's activated quantities (the skip test
a = min(0.99, alpha exp(max(-m/2, -50))) >= cutoff of Algorithm 2); pairs within FP32
rounding of the cutoff may be decided differently, hence the small slack.  The sweep counts
must bound the contributing pairs, come in whole warps, and the list length must match the
binning's own count.
"""
import numpy as np
import pytest

import oracle
from paper_2511_15022_gb300 import inputs
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

CASES = {
    "ragged-100x120-rgb": inputs.custom(100, 120, 1500, wavelengths_m=(638e-9, 520e-9, 450e-9),
                                        z_m=(0.0, 5e-3), seed=21),
    "odd-75x135-mono": inputs.custom(75, 135, 800, z_m=(3e-3,), seed=22),
}


def brute_force_pairs(params, H, W, cutoff):
    act = oracle.activate(params, W, H)
    mx, my, i00, i01, i11, alpha = act[:, 0], act[:, 1], act[:, 8], act[:, 9], act[:, 10], act[:, 11]
    ys, xs = np.mgrid[0:H, 0:W]
    xs = xs.ravel().astype(np.float64)
    ys = ys.ravel().astype(np.float64)
    count = 0
    for n in range(len(mx)):
        dx = xs - mx[n]
        dy = ys - my[n]
        m = i00[n] * dx * dx + 2.0 * i01[n] * dx * dy + i11[n] * dy * dy
        a = np.minimum(0.99, alpha[n] * np.exp(np.maximum(-0.5 * m, -50.0)))
        count += int(np.count_nonzero(a >= cutoff))
    return count


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


@pytest.mark.parametrize("name", sorted(CASES))
def test_raster_stats_against_brute_force(name, dev):
    from paper_2511_15022_gb300 import cgh
    w = CASES[name]
    p_np = inputs.params_for(w)
    plan = cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, cutoff=w.cutoff,
                    max_gaussians=w.N, device=dev)
    s = plan.raster_stats(to_dev(p_np, dev))
    ref = brute_force_pairs(p_np, w.H, w.W, w.cutoff)
    assert ref > 0
    assert abs(s["contributing_pairs"] - ref) <= 1e-4 * ref + 5, (s, ref)
    assert s["overflow_tiles"] == 0
    assert s["tile_pairs"] == plan.status()["pairs"]
    assert s["fwd_lane_slots"] % 32 == 0 and s["bwd_lane_slots"] % 32 == 0
    assert s["fwd_lane_slots"] >= s["contributing_pairs"]
    assert s["bwd_lane_slots"] >= s["contributing_pairs"]
    assert 0 < s["region_pairs"] <= s["tile_pairs"]
    # the backward sweep of a region never evaluates more lane slots than the forward blocks
    # plus the rounding of each (Gaussian, region) pair up to a whole warp
    assert s["bwd_lane_slots"] <= s["fwd_lane_slots"] + 32 * s["region_pairs"]
