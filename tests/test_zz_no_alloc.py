"""The allocation-free forward raster (cgh_raster_fwd_noalloc) against the planned entry
point.  It serves callers that may not allocate device memory, so it keeps its scratch in a
fixed device array inside the library; this checks that two calls in a row (the second
reusing the array as the first left it) give the same field as cgh_raster_fwd, and that
inputs beyond the fixed limits are refused with a message.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2511_15022_gb300 import inputs
from tests.gpu_util import c64, rel_l2, to_dev

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-4


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def test_noalloc_matches_planned_raster_on_two_calls(dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    lib = cgh.load()
    w = inputs.custom(100, 120, 1500, wavelengths_m=(638e-9, 520e-9, 450e-9), z_m=(0.0,),
                      seed=71)
    p = to_dev(inputs.params_for(w), dev)
    plan = cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, cutoff=w.cutoff,
                    max_gaussians=w.N, device=dev)
    ref = c64(plan.raster_fwd(p))
    prm = cgh._Params(w.N, *[ctypes.c_void_p(p[k].data_ptr()) for k in cgh.PARAM_KEYS])
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full((w.C, w.H, w.W), complex(7.0, -7.0), dtype=torch.complex64, device=dev)
        st = lib.cgh_raster_fwd_noalloc(w.H, w.W, w.C, w.cutoff, ctypes.byref(prm),
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0, lib.cgh_last_error_string()
        torch.cuda.synchronize()
        assert rel_l2(c64(out), ref) < FIELD_TOL


def test_noalloc_at_its_tile_limit(dev):
    """2048 x 2048 pixels, the largest grid the fixed array takes (16384 tiles: the tile scan
    then needs more than 48 KB of shared memory), on two calls in a row."""
    import torch
    from paper_2511_15022_gb300 import cgh
    w = inputs.custom(2048, 2048, 40000, wavelengths_m=(638e-9, 520e-9), z_m=(0.0,), seed=73)
    p = to_dev(inputs.params_for(w), dev)
    plan = cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, cutoff=w.cutoff,
                    max_gaussians=w.N, device=dev)
    ref = c64(plan.raster_fwd(p))
    for _ in range(2):
        U = cgh.raster_fwd_noalloc(p, w.H, w.W, w.cutoff)
        torch.cuda.synchronize()
        assert rel_l2(c64(U), ref) < FIELD_TOL


def test_noalloc_refuses_inputs_beyond_its_scratch(dev):
    import torch
    from paper_2511_15022_gb300 import cgh
    lib = cgh.load()
    prm = cgh._Params(70000, *[ctypes.c_void_p(0)] * 6)
    out = torch.empty(1, dtype=torch.complex64, device=dev)
    st = lib.cgh_raster_fwd_noalloc(64, 64, 1, 1 / 255, ctypes.byref(prm),
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert st == 7 and b"65536" in lib.cgh_last_error_string()
    prm = cgh._Params(0, *[ctypes.c_void_p(0)] * 6)
    st = lib.cgh_raster_fwd_noalloc(4096, 4096, 1, 1 / 255, ctypes.byref(prm),
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert st == 5 and b"16384" in lib.cgh_last_error_string()


def test_noalloc_python_binding(dev):
    """The binding of the same name marshals to the C entry point and reports its errors."""
    from paper_2511_15022_gb300 import cgh
    w = inputs.custom(40, 60, 200, z_m=(0.0,), seed=72)
    p = to_dev(inputs.params_for(w), dev)
    plan = cgh.Plan(w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, cutoff=w.cutoff,
                    max_gaussians=w.N, device=dev)
    U = cgh.raster_fwd_noalloc(p, w.H, w.W, w.cutoff)
    assert rel_l2(c64(U), c64(plan.raster_fwd(p))) < FIELD_TOL
    with pytest.raises(cgh.CGHError, match="16384"):
        cgh.raster_fwd_noalloc(p, 4096, 4096, w.cutoff)
