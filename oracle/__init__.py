"""FP64 CPU oracle for complex-valued 2D Gaussian holograms (arXiv 2511.15022).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the product path (``paper_2511_15022_gb300``)
never does and shares no code with it.

The arithmetic lives in ``cgh_oracle.c`` (plain C, FP64, OpenMP over pixels / Gaussians /
FFT lines); this module only compiles it with gcc and marshals numpy arrays through ctypes.
Complex fields are numpy ``complex128`` arrays; a gradient w.r.t. a complex field holds
``dL/dRe + 1j * dL/dIm`` (the convention of the paper's supplementary gradients, Suppl.
"Gradient Flow Overview").

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  raster_fwd    pinned: single-Gaussian closed form, Poisson-summation mass, closed-form
                Fourier transform, symmetries, linearity, cutoff semantics.
  raster_bwd    pinned: central finite differences of raster_fwd (smooth mode), adjoint
                identity <J v, dU> = <v, J^T dU>.
  fft1d/fft2d   pinned: direct DFT (independent loop), impulse/constant, Parseval,
                round trip, numpy.fft.
  blasm_fwd/bwd pinned: z = 0 identity, Parseval (unmasked), z/-z round trip on the
                padded grid, plane-wave eigenmode, composition d1 + d2, band-limit mask
                count from the closed form, adjoint dot-product identity.
  mse_loss/psnr pinned: closed forms, finite differences.
  adam          pinned: hand-iterated scalar recurrence, torch.optim.Adam (CPU).
  recon_loss    pinned: sum of three intensity MSEs of transformed inputs (through the pinned
                mse_loss), finite differences, closed form, no-mask case.
  adan          pinned: equals the pinned Adam with beta2 = 0, constant-gradient closed
                form, gradient-scale invariance, weight decay.
  (encoder_ref.py and poh_ref.py carry their own pin lists.)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cgh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcgh_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile ``cgh_oracle.c`` into ``oracle/_build/libcgh_oracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i, d, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        lib.orc_activate.argtypes = [i, i, i, _dp, _dp, _dp, _dp, _dp]
        lib.orc_raster_fwd.argtypes = [i, i, i, i, _dp, _dp, _dp, _dp, _dp, _dp, d, i, _i64p, _dp]
        lib.orc_raster_bwd.argtypes = [i, i, i, i, _dp, _dp, _dp, _dp, _dp, _dp, d, _dp, i, _i64p,
                                       _dp, _dp, _dp, _dp, _dp, _dp]
        lib.orc_dft1d.argtypes = [i, _dp, i64, i]
        lib.orc_fft1d.argtypes = [i, _dp, i64, i]
        lib.orc_fft2d.argtypes = [i, i, _dp, i]
        lib.orc_blasm_transfer.argtypes = [i, i, d, d, d, d, _dp]
        lib.orc_blasm_fwd.argtypes = [i, i, i, i, i, _dp, d, _dp, d, _dp, _dp]
        lib.orc_blasm_bwd.argtypes = [i, i, i, i, i, _dp, d, _dp, d, _dp, _dp]
        lib.orc_mse_loss.argtypes = [i, i, i, i, _dp, _dp, _dp]
        lib.orc_mse_loss.restype = d
        lib.orc_recon_loss.argtypes = [i, i, i, i, _dp, _dp, ctypes.c_void_p, _dp]
        lib.orc_recon_loss.restype = d
        lib.orc_psnr.argtypes = [i, i, i, i, _dp, _dp]
        lib.orc_psnr.restype = d
        lib.orc_adam.argtypes = [i64, _dp, _dp, _dp, _dp, d, d, d, d, i]
        lib.orc_adan.argtypes = [i64, _dp, _dp, _dp, _dp, _dp, _dp, d, d, d, d, d, d, i]
        lib.orc_num_threads.restype = i
        lib.orc_set_num_threads.argtypes = [i]
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _iptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_i64p)


PARAM_KEYS = ("xy_raw", "s_raw", "theta", "amp", "phase", "alpha_raw")


def _params64(p: dict):
    return {k: _f64(p[k]) for k in PARAM_KEYS}


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def activate(params: dict, W: int, H: int) -> np.ndarray:
    """Activated quantities [N, 12]: mx, my, sx, sy, theta, S00, S01, S11, i00, i01, i11,
    alpha (Suppl. activation, covariance and inversion formulas)."""
    p = _params64(params)
    N = p["theta"].shape[0]
    out = np.zeros((N, 12), np.float64)
    _load().orc_activate(N, W, H, _ptr(p["xy_raw"]), _ptr(p["s_raw"]), _ptr(p["theta"]),
                         _ptr(p["alpha_raw"]), _ptr(out))
    return out


def raster_fwd(params: dict, H: int, W: int, cutoff: float = 1.0 / 255.0,
               pix_idx=None) -> np.ndarray:
    """Brute-force complex rasterisation (Algorithm 2).  Returns complex128 [C, H, W], or
    [C, len(pix_idx)] for a list of linear pixel indices y * W + x."""
    p = _params64(params)
    N, C = p["amp"].shape
    if pix_idx is None:
        U = np.zeros((C, H, W), np.complex128)
        npix, idx = 0, None
    else:
        idx = np.ascontiguousarray(np.asarray(pix_idx, dtype=np.int64))
        npix = idx.shape[0]
        U = np.zeros((C, npix), np.complex128)
    _load().orc_raster_fwd(H, W, C, N, _ptr(p["xy_raw"]), _ptr(p["s_raw"]), _ptr(p["theta"]),
                           _ptr(p["amp"]), _ptr(p["phase"]), _ptr(p["alpha_raw"]),
                           float(cutoff), npix, _iptr(idx), _ptr(U.view(np.float64)))
    return U


def raster_bwd(params: dict, H: int, W: int, dU, cutoff: float = 1.0 / 255.0,
               g_idx=None) -> dict:
    """Analytic backward of the rasteriser (Suppl. gradient items).  dU: complex128
    [C, H, W] holding dL/dRe + 1j dL/dIm.  Returns gradients of the pre-activation
    parameters (for the listed Gaussians only when g_idx is given)."""
    p = _params64(params)
    N, C = p["amp"].shape
    dU = _c128(dU)
    assert dU.shape == (C, H, W)
    if g_idx is None:
        ng, idx = N, None
        cnt = N
    else:
        idx = np.ascontiguousarray(np.asarray(g_idx, dtype=np.int64))
        ng = cnt = idx.shape[0]
    g = {"xy_raw": np.zeros((cnt, 2)), "s_raw": np.zeros((cnt, 2)), "theta": np.zeros(cnt),
         "amp": np.zeros((cnt, C)), "phase": np.zeros((cnt, C)), "alpha_raw": np.zeros(cnt)}
    _load().orc_raster_bwd(H, W, C, N, _ptr(p["xy_raw"]), _ptr(p["s_raw"]), _ptr(p["theta"]),
                           _ptr(p["amp"]), _ptr(p["phase"]), _ptr(p["alpha_raw"]),
                           float(cutoff), _ptr(dU.view(np.float64)), ng, _iptr(idx),
                           _ptr(g["xy_raw"]), _ptr(g["s_raw"]), _ptr(g["theta"]),
                           _ptr(g["amp"]), _ptr(g["phase"]), _ptr(g["alpha_raw"]))
    return g


def dft1d(x, inverse: bool = False) -> np.ndarray:
    """Direct O(N^2) DFT (unnormalised; exp(-2 pi i k n / N) forward)."""
    a = _c128(x).copy()
    _load().orc_dft1d(a.shape[0], _ptr(a.view(np.float64)), 1, int(inverse))
    return a


def fft1d(x, inverse: bool = False) -> np.ndarray:
    """Textbook recursive mixed-radix FFT (unnormalised)."""
    a = _c128(x).copy()
    _load().orc_fft1d(a.shape[0], _ptr(a.view(np.float64)), 1, int(inverse))
    return a


def fft2d(x, inverse: bool = False) -> np.ndarray:
    a = _c128(x).copy()
    ny, nx = a.shape
    _load().orc_fft2d(ny, nx, _ptr(a.view(np.float64)), int(inverse))
    return a


def blasm_transfer(ny: int, nx: int, lam: float, pitch: float, d: float,
                   aperture: float = 0.0) -> np.ndarray:
    """Band-limited transfer function (Algorithm 3) on an ny x nx grid, FFT bin order."""
    out = np.zeros((ny, nx), np.complex128)
    _load().orc_blasm_transfer(ny, nx, float(lam), float(pitch), float(d), float(aperture),
                               _ptr(out.view(np.float64)))
    return out


def blasm_fwd(U0, lambdas, pitch: float, z, pad: int = 2, aperture: float = 0.0) -> np.ndarray:
    """Multi-plane BLASM propagation.  U0 complex [C, H, W] -> Ud complex [L, C, H, W]."""
    U0 = _c128(U0)
    C, H, W = U0.shape
    lam = _f64(lambdas)
    zz = _f64(z)
    L = zz.shape[0]
    Ud = np.zeros((L, C, H, W), np.complex128)
    _load().orc_blasm_fwd(H, W, C, L, int(pad), _ptr(lam), float(pitch), _ptr(zz),
                          float(aperture), _ptr(U0.view(np.float64)), _ptr(Ud.view(np.float64)))
    return Ud


def blasm_bwd(dUd, lambdas, pitch: float, z, pad: int = 2, aperture: float = 0.0) -> np.ndarray:
    """Adjoint BLASM (conj transfer function, summed over planes).  dUd [L, C, H, W]."""
    dUd = _c128(dUd)
    L, C, H, W = dUd.shape
    lam = _f64(lambdas)
    zz = _f64(z)
    dU0 = np.zeros((C, H, W), np.complex128)
    _load().orc_blasm_bwd(H, W, C, L, int(pad), _ptr(lam), float(pitch), _ptr(zz),
                          float(aperture), _ptr(dUd.view(np.float64)), _ptr(dU0.view(np.float64)))
    return dU0


def mse_loss(Ud, target):
    """Multi-plane intensity MSE (Sec. 3.2).  Returns (loss, dL/dUd)."""
    Ud = _c128(Ud)
    L, C, H, W = Ud.shape
    t = _f64(target)
    assert t.shape == (L, C, H, W)
    dUd = np.zeros_like(Ud)
    loss = _load().orc_mse_loss(L, C, H, W, _ptr(Ud.view(np.float64)), _ptr(t),
                                _ptr(dUd.view(np.float64)))
    return float(loss), dUd


def recon_loss(Ud, target, mask=None):
    """Three-term reconstruction loss L_recon (Sec. 3.2) with binary depth masks
    mask [L, H, W] (None: M = 0).  Returns (loss, dL/dUd)."""
    Ud = _c128(Ud)
    L, C, H, W = Ud.shape
    t = _f64(target)
    assert t.shape == (L, C, H, W)
    mptr = None
    if mask is not None:
        m = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
        assert m.shape == (L, H, W)
        mptr = m.ctypes.data_as(ctypes.c_void_p)
    dUd = np.zeros_like(Ud)
    loss = _load().orc_recon_loss(L, C, H, W, _ptr(Ud.view(np.float64)), _ptr(t), mptr,
                                  _ptr(dUd.view(np.float64)))
    return float(loss), dUd


def psnr(Ud, target) -> float:
    Ud = _c128(Ud)
    L, C, H, W = Ud.shape
    t = _f64(target)
    return float(_load().orc_psnr(L, C, H, W, _ptr(Ud.view(np.float64)), _ptr(t)))


def adam(p, g, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One in-place Adam step (PyTorch semantics) on float64 arrays p, m, v."""
    assert p.dtype == np.float64 and p.flags.c_contiguous
    g = _f64(g)
    _load().orc_adam(p.size, _ptr(p), _ptr(g), _ptr(m), _ptr(v), float(lr), float(beta1),
                     float(beta2), float(eps), int(t))


def adan(p, g, m, v, n, gprev, lr, t, beta1=0.98, beta2=0.92, beta3=0.99, eps=1e-8,
         weight_decay=0.0):
    """One in-place Adan step (Sec. 4's optimiser) on float64 arrays p, m, v, n, gprev."""
    for a in (p, m, v, n, gprev):
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == p.shape
    g = _f64(g)
    _load().orc_adan(p.size, _ptr(p), _ptr(g), _ptr(m), _ptr(v), _ptr(n), _ptr(gprev),
                     float(lr), float(beta1), float(beta2), float(beta3), float(eps),
                     float(weight_decay), int(t))


def forward(params: dict, H: int, W: int, lambdas, pitch: float, z, pad: int = 2,
            cutoff: float = 1.0 / 255.0, aperture: float = 0.0):
    """Rasterise then propagate: returns (U0 [C,H,W], Ud [L,C,H,W])."""
    U0 = raster_fwd(params, H, W, cutoff)
    return U0, blasm_fwd(U0, lambdas, pitch, z, pad, aperture)


def step(params: dict, target, H: int, W: int, lambdas, pitch: float, z, pad: int = 2,
         cutoff: float = 1.0 / 255.0, aperture: float = 0.0, g_idx=None, recon_mask=None,
         loss: str = "mse"):
    """One forward + backward pass of the whole hot path (Algorithm 1 body without the
    optimiser): raster -> pad -> multi-plane BLASM -> intensity MSE (or, with
    loss="recon", the three-term L_recon with depth masks recon_mask) -> adjoint BLASM ->
    raster backward.  Returns dict(loss, U0, Ud, dUd, dU0, grads)."""
    U0, Ud = forward(params, H, W, lambdas, pitch, z, pad, cutoff, aperture)
    if loss == "recon":
        loss, dUd = recon_loss(Ud, target, recon_mask)
    else:
        loss, dUd = mse_loss(Ud, target)
    dU0 = blasm_bwd(dUd, lambdas, pitch, z, pad, aperture)
    grads = raster_bwd(params, H, W, dU0, cutoff, g_idx)
    return {"loss": loss, "U0": U0, "Ud": Ud, "dUd": dUd, "dU0": dU0, "grads": grads}
