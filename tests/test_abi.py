"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every
function include/cgh.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "cgh.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cgh_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cgh_raster_fwd", "cgh_raster_bwd", "cgh_blasm_fwd", "cgh_blasm_bwd",
                 "cgh_step", "cgh_plan_create", "cgh_plan_destroy", "cgh_adam_step"):
        assert must in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2511_15022_gb300 import build
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2511_15022_gb300 import cgh
    assert set(cgh.EXPORTS) <= set(declared_functions())
    assert set(declared_functions()) <= set(cgh.EXPORTS)


def test_host_only_calls_without_gpu():
    """Calls that touch no device memory run on a machine without a GPU: error paths,
    kernel names, launch counter."""
    from paper_2511_15022_gb300 import cgh
    lib = cgh.load()
    assert lib.cgh_kernel_count() > 5
    names = [lib.cgh_kernel_name(i).decode() for i in range(lib.cgh_kernel_count())]
    assert "k_raster_fwd" in names and "k_cols_fwd_planes" in names
    assert lib.cgh_launch_count() == 0
    # invalid arguments are rejected before any CUDA call
    h = ctypes.c_void_p()
    lam = (ctypes.c_double * 1)(520e-9)
    z = (ctypes.c_double * 1)(5e-3)
    assert lib.cgh_plan_create(0, 16, 1, 1, 2, lam, 8e-6, z, 0.0, 1 / 255, 10, ctypes.byref(h)) == 1
    assert b"H and W" in lib.cgh_last_error_string()
    assert lib.cgh_plan_create(16, 16, 5, 1, 2, lam, 8e-6, z, 0.0, 1 / 255, 10, ctypes.byref(h)) == 5
    # 7 * 2 = 14 has a prime factor 7: unsupported FFT length
    assert lib.cgh_plan_create(7, 16, 1, 1, 2, lam, 8e-6, z, 0.0, 1 / 255, 10, ctypes.byref(h)) == 5
    assert lib.cgh_raster_fwd(None, None, None, None) == 1
    assert lib.cgh_adam_step(None, 0, 1, 0.9, 0.999, 1e-8, None) == 1


def test_noalloc_binding_rejects_tensors_on_another_device():
    """The allocation-free raster runs on the current device, which its binding makes the
    parameters' device; an output or a stream on another device is refused before any call."""
    import torch
    from paper_2511_15022_gb300 import cgh
    d0, d1 = torch.device("cuda", 0), torch.device("cuda", 1)
    cgh.check_same_device(d0, [("U_out", d0), ("stream", torch.device("cuda", 0))])
    with pytest.raises(cgh.CGHError, match="U_out is on cuda:1"):
        cgh.check_same_device(d0, [("xy_raw", d0), ("U_out", d1)])
    with pytest.raises(cgh.CGHError, match="stream"):
        cgh.check_same_device(d1, [("stream", d0)])
