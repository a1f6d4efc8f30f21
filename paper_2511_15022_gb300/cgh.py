"""Thin Python binding of libcgh (include/cgh.h): argument marshalling only.

Every array is a CUDA torch tensor whose pointer is handed to the C ABI; all arithmetic
runs in the library's sm_103a kernels.  There is no CPU fallback: if the library or a GPU
is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import torch

from . import build as _build

PARAM_KEYS = ("xy_raw", "s_raw", "theta", "amp", "phase", "alpha_raw")

_lib = None


class CGHError(RuntimeError):
    pass


class _Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32)] + [(k, ctypes.c_void_p) for k in PARAM_KEYS]


class _Grads(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in PARAM_KEYS]


class _Tuning(ctypes.Structure):
    _fields_ = [("col_block", ctypes.c_int32), ("row_block", ctypes.c_int32),
                ("fft_threads", ctypes.c_int32), ("pair_capacity_per_gaussian", ctypes.c_int32),
                ("fft_kernels", ctypes.c_int32), ("identity_planes", ctypes.c_int32)]


class _AdanGroup(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p),
                ("exp_avg", ctypes.c_void_p), ("exp_avg_diff", ctypes.c_void_p),
                ("exp_avg_sq", ctypes.c_void_p), ("prev_grad", ctypes.c_void_p),
                ("count", ctypes.c_int64), ("lr", ctypes.c_float)]


class _AdamGroup(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p),
                ("exp_avg", ctypes.c_void_p), ("exp_avg_sq", ctypes.c_void_p),
                ("count", ctypes.c_int64), ("lr", ctypes.c_float)]


EXPORTS = ("cgh_plan_create", "cgh_plan_destroy", "cgh_plan_workspace_bytes",
           "cgh_plan_set_workspace", "cgh_plan_set_tuning", "cgh_plan_get_tuning",
           "cgh_plan_band_limits", "cgh_plan_status", "cgh_raster_fwd", "cgh_raster_bwd",
           "cgh_raster_stats",
           "cgh_blasm_fwd", "cgh_blasm_bwd", "cgh_intensity_loss", "cgh_forward_loss",
           "cgh_intensity", "cgh_intensity_bwd", "cgh_plan_identity_planes",
           "cgh_batch_step_persistent", "cgh_batch_persistent_status", "cgh_batch_persistent_test",
           "cgh_batch_persistent_grid",
           "cgh_step", "cgh_step_scaled", "cgh_adam_step", "cgh_launch_count", "cgh_last_error_string",
           "cgh_profile_enable", "cgh_profile_collect", "cgh_kernel_count", "cgh_kernel_name",
           "cgh_raster_fwd_noalloc", "cgh_adam_step_table", "cgh_batch_create",
           "cgh_batch_destroy", "cgh_batch_bind", "cgh_batch_step", "cgh_batch_kernels_per_step",
           "cgh_autotune", "cgh_conv3x3_fwd", "cgh_conv3x3_bwd", "cgh_cast_bf16",
           "cgh_encoder_decode", "cgh_encoder_decode_bwd", "cgh_mse_grad", "cgh_measure_peaks",
           "cgh_plan_set_loss", "cgh_poh_dpac", "cgh_poh_field", "cgh_poh_scratch_bytes",
           "cgh_poh_step", "cgh_adan_step")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcgh.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise CGHError(f"libcgh.so not found at {path}; run paper_2511_15022_gb300/build.py")
    lib = ctypes.CDLL(path)
    vp, i32, i64, f32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    lib.cgh_plan_create.argtypes = [i32, i32, i32, i32, i32, dp, f64, dp, f64, f32, i32,
                                    ctypes.POINTER(vp)]
    lib.cgh_plan_destroy.argtypes = [vp]
    lib.cgh_plan_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.cgh_plan_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    lib.cgh_plan_set_tuning.argtypes = [vp, ctypes.POINTER(_Tuning)]
    lib.cgh_plan_get_tuning.argtypes = [vp, ctypes.POINTER(_Tuning)]
    lib.cgh_plan_band_limits.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.cgh_plan_status.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                    ctypes.POINTER(i32), vp]
    lib.cgh_raster_fwd.argtypes = [vp, ctypes.POINTER(_Params), vp, vp]
    lib.cgh_raster_fwd_noalloc.argtypes = [i32, i32, i32, f32, ctypes.POINTER(_Params), vp, vp]
    lib.cgh_raster_bwd.argtypes = [vp, ctypes.POINTER(_Params), vp, ctypes.POINTER(_Grads), vp]
    lib.cgh_raster_stats.argtypes = [vp, ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_int64), vp]
    lib.cgh_blasm_fwd.argtypes = [vp, vp, vp, vp]
    lib.cgh_blasm_bwd.argtypes = [vp, vp, vp, vp]
    lib.cgh_intensity_loss.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.cgh_intensity.argtypes = [vp, vp, vp, vp]
    lib.cgh_plan_identity_planes.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
    lib.cgh_intensity_bwd.argtypes = [vp, vp, vp, vp, vp]
    lib.cgh_forward_loss.argtypes = [vp, ctypes.POINTER(_Params), vp, vp, vp]
    lib.cgh_step.argtypes = [vp, ctypes.POINTER(_Params), vp, vp, ctypes.POINTER(_Grads), vp]
    lib.cgh_step_scaled.argtypes = [vp, ctypes.POINTER(_Params), vp, vp, ctypes.POINTER(_Grads),
                                    vp, ctypes.c_int32, vp]
    lib.cgh_adam_step.argtypes = [ctypes.POINTER(_AdamGroup), i32, i32, f32, f32, f32, vp]
    lib.cgh_adam_step_table.argtypes = [vp, vp, i32, i64, i32, f32, f32, f32, f32, vp]
    lib.cgh_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]
    lib.cgh_batch_destroy.argtypes = [vp]
    lib.cgh_batch_bind.argtypes = [vp, i32, ctypes.POINTER(_Params), vp, vp, ctypes.POINTER(_Grads)]
    lib.cgh_batch_step.argtypes = [vp, i32, vp]
    lib.cgh_batch_kernels_per_step.argtypes = [vp]
    lib.cgh_batch_kernels_per_step.restype = i64
    lib.cgh_batch_step_persistent.argtypes = [vp, vp]
    lib.cgh_batch_persistent_status.argtypes = [vp, ctypes.POINTER(i32), vp]
    lib.cgh_batch_persistent_test.argtypes = [vp, i32, f64]
    lib.cgh_batch_persistent_grid.argtypes = [vp]
    lib.cgh_batch_persistent_grid.restype = i32
    lib.cgh_autotune.argtypes = [vp, ctypes.POINTER(_Params), vp, ctypes.POINTER(_Grads), vp, i32,
                                 vp, ctypes.POINTER(_Tuning)]
    lib.cgh_conv3x3_fwd.argtypes = [i32, i32, i32, i32, i32, i32, vp, vp, vp, i32, vp, i32, vp]
    lib.cgh_conv3x3_bwd.argtypes = [i32, i32, i32, i32, i32, i32, vp, vp, i32, vp, i32, vp, vp,
                                    vp, vp, vp]
    lib.cgh_cast_bf16.argtypes = [i64, vp, vp, vp]
    lib.cgh_encoder_decode.argtypes = [i32, i32, i32, i32, i32, i32, i32, vp,
                                       ctypes.POINTER(_Grads), vp]
    lib.cgh_encoder_decode_bwd.argtypes = [i32, i32, i32, i32, i32, i32, i32,
                                           ctypes.POINTER(_Grads), vp, vp]
    lib.cgh_mse_grad.argtypes = [i64, vp, vp, f32, i32, vp, vp, vp]
    lib.cgh_plan_set_loss.argtypes = [vp, i32, vp]
    lib.cgh_adan_step.argtypes = [ctypes.POINTER(_AdanGroup), i32, i32, f32, f32, f32, f32, f32, vp]
    lib.cgh_poh_dpac.argtypes = [vp, vp, vp, i32, vp]
    lib.cgh_poh_field.argtypes = [vp, vp, vp, vp]
    lib.cgh_poh_scratch_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.cgh_poh_step.argtypes = [vp, ctypes.POINTER(_Params), vp, vp, f32, f32, vp,
                                 ctypes.POINTER(_Grads), vp, vp, ctypes.c_size_t, vp]
    lib.cgh_measure_peaks.argtypes = [ctypes.POINTER(f64), ctypes.POINTER(f64), vp]
    lib.cgh_launch_count.restype = i64
    lib.cgh_last_error_string.restype = ctypes.c_char_p
    lib.cgh_profile_enable.argtypes = [i32]
    lib.cgh_profile_collect.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    lib.cgh_kernel_count.restype = i32
    lib.cgh_kernel_name.argtypes = [i32]
    lib.cgh_kernel_name.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("cgh_launch_count", "cgh_last_error_string", "cgh_kernel_count",
                        "cgh_kernel_name", "cgh_batch_kernels_per_step",
                        "cgh_batch_persistent_grid"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != 0:
        msg = _lib.cgh_last_error_string().decode(errors="replace")
        raise CGHError(f"{what} failed with status {status}: {msg}")


def _stream(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _need(t: torch.Tensor, dtype: torch.dtype, shape, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise CGHError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise CGHError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise CGHError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise CGHError(f"{name} must be contiguous")


def measure_peaks(stream=None) -> Dict[str, float]:
    """cgh_measure_peaks: FP32 flop/s and MUFU op/s of the current device."""
    lib = load()
    f, u = ctypes.c_double(), ctypes.c_double()
    _check(lib.cgh_measure_peaks(ctypes.byref(f), ctypes.byref(u), ctypes.c_void_p(_stream(stream))),
           "cgh_measure_peaks")
    return {"fp32_flops_per_s": f.value, "sfu_ops_per_s": u.value}


def launch_count() -> int:
    return int(load().cgh_launch_count())


def profile_enable(on: bool = True) -> None:
    """Start (or stop) per-kernel CUDA-event timing inside the library."""
    lib = load()
    _check(lib.cgh_profile_enable(1 if on else 0), "cgh_profile_enable")


def profile_collect() -> Dict[str, dict]:
    """Per-kernel {ms, launches} since the last collect (waits for the recorded events)."""
    lib = load()
    n = int(lib.cgh_kernel_count())
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check(lib.cgh_profile_collect(ms, cnt), "cgh_profile_collect")
    return {lib.cgh_kernel_name(i).decode(): {"ms": float(ms[i]), "launches": int(cnt[i])}
            for i in range(n) if cnt[i] > 0}


class Plan:
    """One hologram geometry: H x W pixels, C wavelengths, L planes (cgh_plan_create)."""

    def __init__(self, H: int, W: int, wavelengths_m: Sequence[float], pitch_m: float,
                 z_m: Sequence[float], pad: int = 2, aperture: float = 0.0,
                 cutoff: float = 1.0 / 255.0, max_gaussians: int = 1 << 16,
                 device: Optional[torch.device] = None, tuning: Optional[dict] = None):
        lib = load()
        self.H, self.W = int(H), int(W)
        self.C, self.L = len(wavelengths_m), len(z_m)
        self.wavelengths_m = tuple(float(v) for v in wavelengths_m)
        self.z_m = tuple(float(v) for v in z_m)
        self.pitch_m, self.pad, self.cutoff = float(pitch_m), int(pad), float(cutoff)
        self.aperture = float(aperture)
        self.max_gaussians = int(max_gaussians)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        lam = (ctypes.c_double * self.C)(*self.wavelengths_m)
        zz = (ctypes.c_double * self.L)(*self.z_m)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.cgh_plan_create(self.H, self.W, self.C, self.L, self.pad, lam,
                                       self.pitch_m, zz, self.aperture, self.cutoff,
                                       self.max_gaussians, ctypes.byref(h)), "cgh_plan_create")
        self._h = h
        # bumped by every call that may bin Gaussians into the workspace: a caller that saw
        # the same value before and after its own calls knows the binning is still theirs
        self.bin_generation = 0
        self._ws = None
        if tuning:
            self.set_tuning(**tuning)
        self._attach_workspace()

    def _attach_workspace(self):
        n = ctypes.c_size_t()
        _check(_lib.cgh_plan_workspace_bytes(self._h, ctypes.byref(n)), "workspace_bytes")
        if self._ws is None or self._ws.numel() < n.value:
            self._ws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):  # the library zeroes status words on this device
            _check(_lib.cgh_plan_set_workspace(self._h, ctypes.c_void_p(self._ws.data_ptr()),
                                               self._ws.numel()), "set_workspace")

    @property
    def workspace_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(_lib.cgh_plan_workspace_bytes(self._h, ctypes.byref(n)), "workspace_bytes")
        return int(n.value)

    def set_tuning(self, col_block=0, row_block=0, fft_threads=0, pair_capacity_per_gaussian=0,
                   fft_kernels=0, identity_planes=0):
        t = _Tuning(col_block, row_block, fft_threads, pair_capacity_per_gaussian, fft_kernels,
                    identity_planes)
        with torch.cuda.device(self.device):
            _check(_lib.cgh_plan_set_tuning(self._h, ctypes.byref(t)), "set_tuning")
        if self._ws is not None:
            self._attach_workspace()

    # -- phase-only hologram conversion (Sec. 3.3)
    def poh_dpac(self, U0, mode: str = "double", out=None, stream=None) -> torch.Tensor:
        """cgh_poh_dpac: smooth POH exp(j phi_DPAC) of a complex field [C, H, W]; mode
        'double' (double-phase amplitude coding) or 'printed' (the formula as printed)."""
        _need(U0, torch.complex64, (self.C, self.H, self.W), "U0")
        out = out if out is not None else torch.empty_like(U0)
        _need(out, torch.complex64, (self.C, self.H, self.W), "H_out")
        _check(_lib.cgh_poh_dpac(self._h, ctypes.c_void_p(U0.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), {"printed": 0, "double": 1}[mode],
                                 ctypes.c_void_p(_stream(stream))), "cgh_poh_dpac")
        return out

    def poh_field(self, phi, out=None, stream=None) -> torch.Tensor:
        """cgh_poh_field: exp(j phi) for a phase field [C, H, W]."""
        _need(phi, torch.float32, (self.C, self.H, self.W), "phi")
        out = out if out is not None else torch.empty(phi.shape, dtype=torch.complex64,
                                                      device=phi.device)
        _check(_lib.cgh_poh_field(self._h, ctypes.c_void_p(phi.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream(stream))),
               "cgh_poh_field")
        return out

    def poh_step(self, params, phi, target, lambda_comp=0.1, lambda_field=0.01, grads=None,
                 dphi=None, loss_out=None, stream=None):
        """cgh_poh_step: joint random-POH conversion pass.  Returns (loss, grads, dphi)."""
        prm = self._params(params)
        _need(phi, torch.float32, (self.C, self.H, self.W), "phi")
        _need(target, torch.float32, (self.L, self.C, self.H, self.W), "target")
        g = grads if grads is not None else self.empty_grads(prm.N)
        gs = self._grads(g, prm.N)
        dphi = dphi if dphi is not None else torch.empty_like(phi)
        _need(dphi, torch.float32, (self.C, self.H, self.W), "dphi")
        loss = loss_out if loss_out is not None else torch.empty(1, device=self.device)
        n = ctypes.c_size_t()
        _check(_lib.cgh_poh_scratch_bytes(self._h, ctypes.byref(n)), "cgh_poh_scratch_bytes")
        if getattr(self, "_poh_scratch", None) is None or self._poh_scratch.numel() < n.value:
            self._poh_scratch = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        _check(_lib.cgh_poh_step(self._h, ctypes.byref(prm), ctypes.c_void_p(phi.data_ptr()),
                                 ctypes.c_void_p(target.data_ptr()), float(lambda_comp),
                                 float(lambda_field), ctypes.c_void_p(loss.data_ptr()),
                                 ctypes.byref(gs), ctypes.c_void_p(dphi.data_ptr()),
                                 ctypes.c_void_p(self._poh_scratch.data_ptr()), n.value,
                                 ctypes.c_void_p(_stream(stream))), "cgh_poh_step")
        return loss, g, dphi

    def set_loss(self, kind: str = "mse", mask=None):
        """cgh_plan_set_loss: 'mse' (L_MSE) or 'recon' (three-term L_recon with the binary
        depth masks `mask`, a CUDA uint8 tensor [L, H, W], or None for M = 0)."""
        k = {"mse": 0, "recon": 1}[kind]
        if mask is not None:
            _need(mask, torch.uint8, (self.L, self.H, self.W), "mask")
        self._mask = mask  # the plan reads it at every later call
        _check(_lib.cgh_plan_set_loss(self._h, k, ctypes.c_void_p(mask.data_ptr()) if mask is not None
                                      else ctypes.c_void_p(0)), "cgh_plan_set_loss")

    @property
    def identity_planes(self) -> tuple:
        """Indices of the planes whose propagation is the identity (cgh_plan_identity_planes)."""
        m = ctypes.c_uint32()
        _check(_lib.cgh_plan_identity_planes(self._h, ctypes.byref(m)), "cgh_plan_identity_planes")
        return tuple(l for l in range(self.L) if (m.value >> l) & 1)

    def get_tuning(self) -> dict:
        t = _Tuning()
        _check(_lib.cgh_plan_get_tuning(self._h, ctypes.byref(t)), "get_tuning")
        return {k: getattr(t, k) for k, _ in _Tuning._fields_}

    def band_limits(self):
        kx = (ctypes.c_int32 * (self.C * self.L))()
        ky = (ctypes.c_int32 * (self.C * self.L))()
        _check(_lib.cgh_plan_band_limits(self._h, kx, ky), "band_limits")
        return list(kx), list(ky)

    def status(self, stream=None) -> dict:
        pairs, ov, nf = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.cgh_plan_status(self._h, ctypes.byref(pairs), ctypes.byref(ov),
                                    ctypes.byref(nf), ctypes.c_void_p(_stream(stream))), "status")
        return {"pairs": int(pairs.value), "overflow": bool(ov.value), "nonfinite": bool(nf.value)}

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.cgh_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- marshalling helpers
    def _params(self, p: Dict[str, torch.Tensor]) -> _Params:
        N = int(p["theta"].shape[0])
        shapes = {"xy_raw": (N, 2), "s_raw": (N, 2), "theta": (N,), "amp": (N, self.C),
                  "phase": (N, self.C), "alpha_raw": (N,)}
        for k in PARAM_KEYS:
            _need(p[k], torch.float32, shapes[k], k)
        # every call that takes parameters may rebin them in the workspace
        self.bin_generation += 1
        return _Params(N, *[ctypes.c_void_p(p[k].data_ptr()) for k in PARAM_KEYS])

    def empty_grads(self, N: int) -> Dict[str, torch.Tensor]:
        d = self.device
        return {"xy_raw": torch.empty(N, 2, device=d), "s_raw": torch.empty(N, 2, device=d),
                "theta": torch.empty(N, device=d), "amp": torch.empty(N, self.C, device=d),
                "phase": torch.empty(N, self.C, device=d), "alpha_raw": torch.empty(N, device=d)}

    def _grads(self, g: Dict[str, torch.Tensor], N: int) -> _Grads:
        shapes = {"xy_raw": (N, 2), "s_raw": (N, 2), "theta": (N,), "amp": (N, self.C),
                  "phase": (N, self.C), "alpha_raw": (N,)}
        for k in PARAM_KEYS:
            _need(g[k], torch.float32, shapes[k], "grad " + k)
        return _Grads(*[ctypes.c_void_p(g[k].data_ptr()) for k in PARAM_KEYS])

    # -- entry points (same names as the C ABI)
    def raster_fwd(self, params, out=None, stream=None) -> torch.Tensor:
        prm = self._params(params)
        U = out if out is not None else torch.empty(self.C, self.H, self.W, dtype=torch.complex64,
                                                    device=self.device)
        _need(U, torch.complex64, (self.C, self.H, self.W), "U_out")
        _check(_lib.cgh_raster_fwd(self._h, ctypes.byref(prm), ctypes.c_void_p(U.data_ptr()),
                                   ctypes.c_void_p(_stream(stream))), "cgh_raster_fwd")
        return U

    def raster_stats(self, params, stream=None) -> dict:
        """cgh_raster_stats: work counters of the forward and backward sweeps."""
        prm = self._params(params)
        c = (ctypes.c_int64 * 6)()
        with torch.cuda.device(self.device):
            _check(_lib.cgh_raster_stats(self._h, ctypes.byref(prm), c,
                                         ctypes.c_void_p(_stream(stream))), "cgh_raster_stats")
        keys = ("fwd_lane_slots", "contributing_pairs", "bwd_lane_slots", "region_pairs",
                "tile_pairs", "overflow_tiles")
        return {k: int(c[i]) for i, k in enumerate(keys)}

    def raster_bwd(self, params, dU, grads=None, stream=None) -> Dict[str, torch.Tensor]:
        prm = self._params(params)
        _need(dU, torch.complex64, (self.C, self.H, self.W), "dU")
        g = grads if grads is not None else self.empty_grads(prm.N)
        gs = self._grads(g, prm.N)
        _check(_lib.cgh_raster_bwd(self._h, ctypes.byref(prm), ctypes.c_void_p(dU.data_ptr()),
                                   ctypes.byref(gs), ctypes.c_void_p(_stream(stream))),
               "cgh_raster_bwd")
        return g

    def blasm_fwd(self, U0, out=None, stream=None) -> torch.Tensor:
        _need(U0, torch.complex64, (self.C, self.H, self.W), "U0")
        Ud = out if out is not None else torch.empty(self.L, self.C, self.H, self.W,
                                                     dtype=torch.complex64, device=self.device)
        _need(Ud, torch.complex64, (self.L, self.C, self.H, self.W), "Ud_out")
        _check(_lib.cgh_blasm_fwd(self._h, ctypes.c_void_p(U0.data_ptr()),
                                  ctypes.c_void_p(Ud.data_ptr()), ctypes.c_void_p(_stream(stream))),
               "cgh_blasm_fwd")
        return Ud

    def blasm_bwd(self, dUd, out=None, stream=None) -> torch.Tensor:
        _need(dUd, torch.complex64, (self.L, self.C, self.H, self.W), "dUd")
        dU0 = out if out is not None else torch.empty(self.C, self.H, self.W,
                                                      dtype=torch.complex64, device=self.device)
        _need(dU0, torch.complex64, (self.C, self.H, self.W), "dU0_out")
        _check(_lib.cgh_blasm_bwd(self._h, ctypes.c_void_p(dUd.data_ptr()),
                                  ctypes.c_void_p(dU0.data_ptr()), ctypes.c_void_p(_stream(stream))),
               "cgh_blasm_bwd")
        return dU0

    def intensity_loss(self, Ud, target, want_grad=True, stream=None):
        _need(Ud, torch.complex64, (self.L, self.C, self.H, self.W), "Ud")
        _need(target, torch.float32, (self.L, self.C, self.H, self.W), "target")
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        dUd = torch.empty_like(Ud) if want_grad else None
        _check(_lib.cgh_intensity_loss(self._h, ctypes.c_void_p(Ud.data_ptr()),
                                       ctypes.c_void_p(target.data_ptr()),
                                       ctypes.c_void_p(loss.data_ptr()),
                                       ctypes.c_void_p(dUd.data_ptr() if dUd is not None else 0),
                                       ctypes.c_void_p(_stream(stream))), "cgh_intensity_loss")
        return loss, dUd

    def intensity(self, Ud, out=None, stream=None) -> torch.Tensor:
        """cgh_intensity: I = |Ud|^2, float32 [L, C, H, W]."""
        shape = (self.L, self.C, self.H, self.W)
        _need(Ud, torch.complex64, shape, "Ud")
        I = out if out is not None else torch.empty(shape, dtype=torch.float32, device=self.device)
        _need(I, torch.float32, shape, "I_out")
        _check(_lib.cgh_intensity(self._h, ctypes.c_void_p(Ud.data_ptr()),
                                  ctypes.c_void_p(I.data_ptr()), ctypes.c_void_p(_stream(stream))),
               "cgh_intensity")
        return I

    def intensity_bwd(self, Ud, dI, out=None, stream=None) -> torch.Tensor:
        """cgh_intensity_bwd: dL/dUd = 2 dL/dI Ud, complex64 [L, C, H, W]."""
        shape = (self.L, self.C, self.H, self.W)
        _need(Ud, torch.complex64, shape, "Ud")
        _need(dI, torch.float32, shape, "dI")
        dUd = out if out is not None else torch.empty(shape, dtype=torch.complex64, device=self.device)
        _need(dUd, torch.complex64, shape, "dUd_out")
        _check(_lib.cgh_intensity_bwd(self._h, ctypes.c_void_p(Ud.data_ptr()),
                                      ctypes.c_void_p(dI.data_ptr()), ctypes.c_void_p(dUd.data_ptr()),
                                      ctypes.c_void_p(_stream(stream))), "cgh_intensity_bwd")
        return dUd

    def forward_loss(self, params, target, loss_out=None, stream=None) -> torch.Tensor:
        prm = self._params(params)
        _need(target, torch.float32, (self.L, self.C, self.H, self.W), "target")
        loss = loss_out if loss_out is not None else torch.empty(1, dtype=torch.float32,
                                                                 device=self.device)
        _check(_lib.cgh_forward_loss(self._h, ctypes.byref(prm), ctypes.c_void_p(target.data_ptr()),
                                     ctypes.c_void_p(loss.data_ptr()),
                                     ctypes.c_void_p(_stream(stream))), "cgh_forward_loss")
        return loss

    def autotune(self, params, target, iters: int = 5, stream=None) -> dict:
        """cgh_autotune: time every valid block shape on this data and keep the fastest."""
        prm = self._params(params)
        _need(target, torch.float32, (self.L, self.C, self.H, self.W), "target")
        g = self.empty_grads(prm.N)
        gs = self._grads(g, prm.N)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        best = _Tuning()
        _check(_lib.cgh_autotune(self._h, ctypes.byref(prm), ctypes.c_void_p(target.data_ptr()),
                                 ctypes.byref(gs), ctypes.c_void_p(loss.data_ptr()), int(iters),
                                 ctypes.c_void_p(_stream(stream)), ctypes.byref(best)),
               "cgh_autotune")
        return {k: getattr(best, k) for k, _ in _Tuning._fields_}

    def step(self, params, target, grads=None, loss_out=None, stream=None, grad_scale=None,
             reuse_binning: bool = False):
        """Fused forward + backward (cgh_step).  Returns (loss[1], grads).

        grad_scale (a one-element float32 device tensor) multiplies every gradient and
        reuse_binning keeps the workspace's binning of these parameters (cgh_step_scaled)."""
        prm = self._params(params)
        _need(target, torch.float32, (self.L, self.C, self.H, self.W), "target")
        g = grads if grads is not None else self.empty_grads(prm.N)
        gs = self._grads(g, prm.N)
        loss = loss_out if loss_out is not None else torch.empty(1, dtype=torch.float32,
                                                                 device=self.device)
        if grad_scale is None and not reuse_binning:
            _check(_lib.cgh_step(self._h, ctypes.byref(prm), ctypes.c_void_p(target.data_ptr()),
                                 ctypes.c_void_p(loss.data_ptr()), ctypes.byref(gs),
                                 ctypes.c_void_p(_stream(stream))), "cgh_step")
            return loss, g
        if grad_scale is not None:
            if (grad_scale.dtype != torch.float32 or grad_scale.numel() != 1
                    or grad_scale.device != self.device):
                raise ValueError("grad_scale must be one float32 element on the plan's device")
        _check(_lib.cgh_step_scaled(self._h, ctypes.byref(prm), ctypes.c_void_p(target.data_ptr()),
                                    ctypes.c_void_p(loss.data_ptr()), ctypes.byref(gs),
                                    ctypes.c_void_p(grad_scale.data_ptr() if grad_scale is not None
                                                    else 0),
                                    1 if reuse_binning else 0,
                                    ctypes.c_void_p(_stream(stream))), "cgh_step_scaled")
        return loss, g


def raster_fwd_noalloc(params, H: int, W: int, cutoff: float = 1.0 / 255.0, out=None,
                       stream=None) -> torch.Tensor:
    """cgh_raster_fwd_noalloc: the forward raster with no plan and no device allocation
    inside the library (fixed scratch; N <= 65536, at most 16384 16x16 tiles)."""
    lib = load()
    N = int(params["theta"].shape[0])
    C = int(params["amp"].shape[1])
    shapes = {"xy_raw": (N, 2), "s_raw": (N, 2), "theta": (N,), "amp": (N, C),
              "phase": (N, C), "alpha_raw": (N,)}
    for k in PARAM_KEYS:
        _need(params[k], torch.float32, shapes[k], k)
    dev = params["theta"].device
    check_same_device(dev, [(k, params[k].device) for k in PARAM_KEYS]
                      + ([("U_out", out.device)] if out is not None else [])
                      + ([("stream", stream.device)] if stream is not None else []))
    prm = _Params(N, *[ctypes.c_void_p(params[k].data_ptr()) for k in PARAM_KEYS])
    U = out if out is not None else torch.empty(C, H, W, dtype=torch.complex64, device=dev)
    _need(U, torch.complex64, (C, H, W), "U_out")
    # the entry point works on the current device: make it the parameters' device
    with torch.cuda.device(dev):
        _check(lib.cgh_raster_fwd_noalloc(int(H), int(W), C, float(cutoff), ctypes.byref(prm),
                                          ctypes.c_void_p(U.data_ptr()),
                                          ctypes.c_void_p(_stream(stream))),
               "cgh_raster_fwd_noalloc")
    return U


def check_same_device(device, named_devices) -> None:
    """Raise CGHError unless every (name, torch.device) pair is on `device` (a device without
    an index means the current one only when `device` has none either)."""
    want = torch.device(device)
    for name, d in named_devices:
        d = torch.device(d)
        if d.type != want.type or (d.index != want.index):
            raise CGHError(f"{name} is on {d}, but the parameters are on {want}")


def adam_step(groups, step: int, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """Fused Adam over up to 8 groups: each group is (param, grad, exp_avg, exp_avg_sq, lr)."""
    lib = load()
    arr = (_AdamGroup * len(groups))()
    for i, (p, g, m, v, lr) in enumerate(groups):
        for t, name in ((p, "param"), (g, "grad"), (m, "exp_avg"), (v, "exp_avg_sq")):
            _need(t, torch.float32, tuple(p.shape), name)
        arr[i] = _AdamGroup(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), p.numel(),
                            float(lr))
    _check(lib.cgh_adam_step(arr, len(groups), int(step), float(beta1), float(beta2), float(eps),
                             ctypes.c_void_p(_stream(stream))), "cgh_adam_step")


def adan_step(groups, step: int, beta1=0.98, beta2=0.92, beta3=0.99, eps=1e-8,
              weight_decay=0.0, stream=None):
    """Adan over up to 8 groups (cgh_adan_step): each group is
    (param, grad, exp_avg, exp_avg_diff, exp_avg_sq, prev_grad, lr)."""
    lib = load()
    arr = (_AdanGroup * len(groups))()
    for i, (p, g, m, v, n, gp, lr) in enumerate(groups):
        for t, name in ((p, "param"), (g, "grad"), (m, "exp_avg"), (v, "exp_avg_diff"),
                        (n, "exp_avg_sq"), (gp, "prev_grad")):
            _need(t, torch.float32, tuple(p.shape), name)
        arr[i] = _AdanGroup(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), n.data_ptr(),
                            gp.data_ptr(), p.numel(), float(lr))
    _check(lib.cgh_adan_step(arr, len(groups), int(step), float(beta1), float(beta2),
                             float(beta3), float(eps), float(weight_decay),
                             ctypes.c_void_p(_stream(stream))), "cgh_adan_step")


class AdamTable:
    """Adam over many parameter groups in one launch (cgh_adam_step_table).  groups is a
    list of (param, exp_avg, exp_avg_sq, grad, lr); the tensors must stay alive."""

    def __init__(self, groups, beta1=0.9, beta2=0.999, eps=1e-8):
        load()
        self.groups = list(groups)
        dev = self.groups[0][0].device
        recs = (_AdamGroup * len(self.groups))()
        offs = [0]
        for i, (p, m, v, g, lr) in enumerate(self.groups):
            for t, name in ((m, "exp_avg"), (v, "exp_avg_sq"), (g, "grad")):
                _need(t, torch.float32, tuple(p.shape), name)
            recs[i] = _AdamGroup(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(),
                                 p.numel(), float(lr))
            offs.append(offs[-1] + p.numel())
        raw = bytes(recs)
        self.table = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(dev)
        self.offsets = torch.tensor(offs, dtype=torch.int64, device=dev)
        self.total = offs[-1]
        self.beta1, self.beta2, self.eps = beta1, beta2, eps
        self.t = 0

    def step(self, lr_scale: float = 1.0, stream=None):
        """One Adam step of every group, learning rates multiplied by lr_scale."""
        self.t += 1
        _check(_lib.cgh_adam_step_table(ctypes.c_void_p(self.table.data_ptr()),
                                        ctypes.c_void_p(self.offsets.data_ptr()),
                                        len(self.groups), self.total, self.t, self.beta1,
                                        self.beta2, self.eps, float(lr_scale),
                                        ctypes.c_void_p(_stream(stream))),
               "cgh_adam_step_table")


class Batch:
    """Independent holograms stepped together (cgh_batch_*): one graph launch per step."""

    def __init__(self, plans):
        load()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(_lib.cgh_batch_create(arr, len(self.plans), ctypes.byref(h)), "cgh_batch_create")
        self._h = h
        self._keep = {}

    def bind(self, i: int, params, target, grads, loss_out):
        plan = self.plans[i]
        prm = plan._params(params)
        gs = plan._grads(grads, prm.N)
        _need(target, torch.float32, (plan.L, plan.C, plan.H, plan.W), "target")
        _need(loss_out, torch.float32, (1,), "loss_out")
        self._keep[i] = (params, target, grads, loss_out)
        _check(_lib.cgh_batch_bind(self._h, int(i), ctypes.byref(prm),
                                   ctypes.c_void_p(target.data_ptr()),
                                   ctypes.c_void_p(loss_out.data_ptr()), ctypes.byref(gs)),
               "cgh_batch_bind")

    def step(self, use_graph: bool = True, stream=None):
        _check(_lib.cgh_batch_step(self._h, 1 if use_graph else 0,
                                   ctypes.c_void_p(_stream(stream))), "cgh_batch_step")

    @property
    def kernels_per_step(self) -> int:
        return int(_lib.cgh_batch_kernels_per_step(self._h))

    def step_persistent(self, stream=None):
        """cgh_batch_step_persistent: the whole batched step as one persistent launch."""
        _check(_lib.cgh_batch_step_persistent(self._h, ctypes.c_void_p(_stream(stream))),
               "cgh_batch_step_persistent")

    def persistent_status(self, stream=None) -> bool:
        """True if a grid-barrier wait of the last persistent step ran out (it then returned
        early; its outputs are not valid)."""
        t = ctypes.c_int32()
        st = _lib.cgh_batch_persistent_status(self._h, ctypes.byref(t),
                                              ctypes.c_void_p(_stream(stream)))
        if st not in (0, 3):
            _check(st, "cgh_batch_persistent_status")
        return bool(t.value)

    def persistent_test(self, skip_barrier: int = -1, timeout_s: float = 0.0):
        """Test hook: CTA 0 skips its arrival at grid barrier `skip_barrier` (-1: off); the
        barrier wait budget in seconds (<= 0: default)."""
        _check(_lib.cgh_batch_persistent_test(self._h, int(skip_barrier), float(timeout_s)),
               "cgh_batch_persistent_test")

    @property
    def persistent_grid(self) -> int:
        return int(_lib.cgh_batch_persistent_grid(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.cgh_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- learned-initialiser layers
def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def conv_out_size(n: int, stride: int) -> int:
    return (n - 1) // stride + 1


def conv3x3_fwd(x_bf16, w_bf16, bias, stride: int, relu: bool, out_f32: bool = False,
                out=None, stream=None):
    """cgh_conv3x3_fwd.  x [B,CI,H,W] bf16, w [CO,CI,3,3] bf16, bias [CO] f32."""
    lib = load()
    B, CI, H, W = x_bf16.shape
    CO = w_bf16.shape[0]
    Ho, Wo = conv_out_size(H, stride), conv_out_size(W, stride)
    _need(x_bf16, torch.bfloat16, (B, CI, H, W), "x")
    _need(w_bf16, torch.bfloat16, (CO, CI, 3, 3), "w")
    _need(bias, torch.float32, (CO,), "bias")
    ydt = torch.float32 if out_f32 else torch.bfloat16
    y = out if out is not None else torch.empty(B, CO, Ho, Wo, device=x_bf16.device, dtype=ydt)
    _need(y, ydt, (B, CO, Ho, Wo), "y")
    _check(lib.cgh_conv3x3_fwd(B, CI, H, W, CO, stride, _ptr(x_bf16), _ptr(w_bf16), _ptr(bias),
                               1 if relu else 0, _ptr(y), 1 if out_f32 else 0,
                               ctypes.c_void_p(_stream(stream))), "cgh_conv3x3_fwd")
    return y


def conv3x3_bwd(x_bf16, w_bf16, y, dy, stride: int, relu: bool, want_dx: bool = True,
                dx=None, dw=None, db=None, stream=None):
    """cgh_conv3x3_bwd: returns (dx or None, dw, db), all f32 (dw, db overwritten)."""
    lib = load()
    B, CI, H, W = x_bf16.shape
    CO = w_bf16.shape[0]
    dev = x_bf16.device
    if want_dx and dx is None:
        dx = torch.empty(B, CI, H, W, device=dev)
    if not want_dx:
        dx = None
    dw = dw if dw is not None else torch.empty(CO, CI, 3, 3, device=dev)
    db = db if db is not None else torch.empty(CO, device=dev)
    _need(x_bf16, torch.bfloat16, (B, CI, H, W), "x")
    _need(w_bf16, torch.bfloat16, (CO, CI, 3, 3), "w")
    yshape = (B, CO, conv_out_size(H, stride), conv_out_size(W, stride))
    if y is not None:
        _need(y, y.dtype, yshape, "y")
        if y.dtype not in (torch.float32, torch.bfloat16):
            raise CGHError("y must be float32 or bfloat16")
    elif relu:
        raise CGHError("relu backward needs the forward output y")
    _need(dy, torch.float32, yshape, "dy")
    if dx is not None:
        _need(dx, torch.float32, (B, CI, H, W), "dx")
    _need(dw, torch.float32, (CO, CI, 3, 3), "dw")
    _need(db, torch.float32, (CO,), "db")
    y_f32 = 1 if (y is not None and y.dtype == torch.float32) else 0
    _check(lib.cgh_conv3x3_bwd(B, CI, H, W, CO, stride, _ptr(x_bf16), _ptr(w_bf16),
                               1 if relu else 0, _ptr(y), y_f32, _ptr(dy), _ptr(dx), _ptr(dw),
                               _ptr(db), ctypes.c_void_p(_stream(stream))), "cgh_conv3x3_bwd")
    return dx, dw, db


def cast_bf16(src, dst=None, stream=None):
    """cgh_cast_bf16: f32 -> bf16 (round to nearest even)."""
    lib = load()
    if not src.is_cuda or src.dtype != torch.float32 or not src.is_contiguous():
        raise CGHError("src must be a contiguous CUDA float32 tensor")
    d = dst if dst is not None else torch.empty(src.shape, dtype=torch.bfloat16, device=src.device)
    _need(d, torch.bfloat16, tuple(src.shape), "dst")
    _check(lib.cgh_cast_bf16(src.numel(), _ptr(src), _ptr(d), ctypes.c_void_p(_stream(stream))),
           "cgh_cast_bf16")
    return d


def param_dict(n: int, C: int, device) -> Dict[str, torch.Tensor]:
    """Empty pre-activation parameter (or gradient) arrays for n Gaussians."""
    return {"xy_raw": torch.empty(n, 2, device=device), "s_raw": torch.empty(n, 2, device=device),
            "theta": torch.empty(n, device=device), "amp": torch.empty(n, C, device=device),
            "phase": torch.empty(n, C, device=device), "alpha_raw": torch.empty(n, device=device)}


def _param_struct(d, n: int, C: int):
    shapes = {"xy_raw": (n, 2), "s_raw": (n, 2), "theta": (n,), "amp": (n, C), "phase": (n, C),
              "alpha_raw": (n,)}
    for k in PARAM_KEYS:
        _need(d[k], torch.float32, shapes[k], k)
    return _Grads(*[_ptr(d[k]) for k in PARAM_KEYS])


def encoder_decode(out, S: int, C: int, H: int, W: int, params=None, stream=None):
    """cgh_encoder_decode: out [B, S*(6+2C), CY, CX] f32 -> parameters of B*CY*CX*S Gaussians."""
    lib = load()
    B, P, CY, CX = out.shape
    if P != S * (6 + 2 * C):
        raise CGHError(f"encoder output has {P} channels, expected {S * (6 + 2 * C)}")
    _need(out, torch.float32, (B, P, CY, CX), "out")
    n = B * CY * CX * S
    p = params if params is not None else param_dict(n, C, out.device)
    st = _param_struct(p, n, C)
    _check(lib.cgh_encoder_decode(B, CY, CX, S, C, H, W, _ptr(out), ctypes.byref(st),
                                  ctypes.c_void_p(_stream(stream))), "cgh_encoder_decode")
    return p


def encoder_decode_bwd(grads, B: int, CY: int, CX: int, S: int, C: int, H: int, W: int,
                       dout=None, stream=None):
    """cgh_encoder_decode_bwd: parameter gradients -> dL/d(encoder output)."""
    lib = load()
    dev = grads["theta"].device
    shape = (B, S * (6 + 2 * C), CY, CX)
    dout = dout if dout is not None else torch.empty(shape, device=dev)
    _need(dout, torch.float32, shape, "dout")
    st = _param_struct(grads, B * CY * CX * S, C)
    _check(lib.cgh_encoder_decode_bwd(B, CY, CX, S, C, H, W, ctypes.byref(st), _ptr(dout),
                                      ctypes.c_void_p(_stream(stream))), "cgh_encoder_decode_bwd")
    return dout


def mse_grad(pred, target, weight: float, grad_out, accumulate: bool = False, loss_accum=None,
             stream=None):
    """cgh_mse_grad: grad_out (+)= 2 w (pred - target); loss_accum += w sum (pred - target)^2."""
    lib = load()
    for t, name in ((pred, "pred"), (target, "target"), (grad_out, "grad")):
        _need(t, torch.float32, tuple(pred.shape), name)
        if not t.is_contiguous():
            raise CGHError(f"{name} must be contiguous")
    if loss_accum is not None:
        _need(loss_accum, torch.float32, (1,), "loss_accum")
    _check(lib.cgh_mse_grad(pred.numel(), _ptr(pred), _ptr(target), float(weight),
                            1 if accumulate else 0, _ptr(grad_out), _ptr(loss_accum),
                            ctypes.c_void_p(_stream(stream))), "cgh_mse_grad")
