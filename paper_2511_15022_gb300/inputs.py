"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the benchmark.

This module draws random numbers only; it holds none of the method's arithmetic (no
rasterisation, propagation or loss).  Parameters are produced directly in the
pre-activation form the method optimises, using the inverse of the activations the paper
states for its own initialisation (Sec. 4: means via atanh(2x/W - 1); Suppl. activation:
s = exp(s_raw) + 0.1, alpha = sigmoid(alpha_raw)).

Recipes (numbers follow the workload descriptions this project measures on):
  * means uniform over [0, W] x [0, H]; each activated scale log-uniform in
    [s_min, s_max] pixels; rotation uniform in [0, pi); amplitude U(0, 1) and phase
    U(0, 2 pi) per channel; alpha_raw = -0.5 (the paper's opacity initialisation).
  * target intensities: per (plane, channel) a sum of isotropic Gaussian blobs with
    sigma U(8, 40) px and peak U(0.3, 1), normalised so the maximum is 1 (smooth
    natural-image stand-in; the paper's DIV2K/focal-stack targets are not available).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

SEED_GAUSSIANS = 1234
SEED_TARGETS = 4321
SEED_PLANTED = 999


@dataclasses.dataclass(frozen=True)
class Workload:
    """One hologram problem: image size, optics and primitive count."""
    name: str
    H: int
    W: int
    wavelengths_m: Sequence[float]
    pitch_m: float
    z_m: Sequence[float]
    N: int
    s_min_px: float = 0.5
    s_max_px: float = 4.0
    pad: int = 2
    cutoff: float = 1.0 / 255.0
    seed: int = SEED_GAUSSIANS

    @property
    def C(self) -> int:
        return len(self.wavelengths_m)

    @property
    def L(self) -> int:
        return len(self.z_m)


def small_256() -> Workload:
    """256x256, one 520 nm channel, 8 um pitch, 2048 Gaussians, one plane at 5 mm."""
    return Workload("small-256x256-C1-L1-N2048", 256, 256, (520e-9,), 8e-6, (5e-3,), 2048,
                    seed=SEED_GAUSSIANS + 0)


def hd_1080p() -> Workload:
    """1080x1920, RGB 638/520/450 nm, 8 um pitch, 200k Gaussians, planes at 0/5/10 mm."""
    return Workload("1080x1920-C3-L3-N200k", 1080, 1920, (638e-9, 520e-9, 450e-9), 8e-6,
                    (0.0, 5e-3, 10e-3), 200_000, seed=SEED_GAUSSIANS + 1)


def uhd_4k(rng_seed: int = SEED_GAUSSIANS + 2) -> Workload:
    """2160x3840, RGB, 1M Gaussians with scales 0.3-8 px, 6 planes z ~ U[0, 20] mm."""
    rng = np.random.default_rng(rng_seed)
    z = tuple(float(v) for v in np.sort(rng.uniform(0.0, 20e-3, size=6)))
    return Workload("2160x3840-C3-L6-N1M", 2160, 3840, (638e-9, 520e-9, 450e-9), 8e-6, z,
                    1_000_000, s_min_px=0.3, s_max_px=8.0, seed=rng_seed)


def custom(H: int, W: int, N: int, wavelengths_m=(520e-9,), z_m=(5e-3,), pitch_m=8e-6,
           s_min_px=0.5, s_max_px=4.0, seed=SEED_GAUSSIANS, cutoff=1.0 / 255.0,
           name: Optional[str] = None) -> Workload:
    return Workload(name or f"{H}x{W}-C{len(wavelengths_m)}-L{len(z_m)}-N{N}", H, W,
                    tuple(wavelengths_m), pitch_m, tuple(z_m), N, s_min_px, s_max_px,
                    seed=seed, cutoff=cutoff)


BATCH_BUCKETS = ((256, 256), (512, 512), (512, 768), (640, 1024), (1024, 1024), (1080, 1920))


def batched_64(seed: int = SEED_GAUSSIANS + 3, count: int = 64) -> List[Workload]:
    """64 independent holograms: sizes uniform over six buckets, N ~ U[5k, 300k],
    L ~ U{1, 2, 3} planes drawn from {0, 5, 10} mm, RGB."""
    rng = np.random.default_rng(seed)
    out = []
    zs = (0.0, 5e-3, 10e-3)
    for i in range(count):
        H, W = BATCH_BUCKETS[int(rng.integers(0, len(BATCH_BUCKETS)))]
        N = int(rng.integers(5_000, 300_001))
        L = int(rng.integers(1, 4))
        z = tuple(sorted(rng.choice(zs, size=L, replace=False).tolist()))
        out.append(Workload(f"batch{i}-{H}x{W}-L{L}-N{N}", H, W, (638e-9, 520e-9, 450e-9),
                            8e-6, z, N, seed=seed * 1000 + i))
    return out


def _draw_means(rng, N: int, H: int, W: int):
    """The first draws of a parameter set: Gaussian means uniform over [0, W] x [0, H]."""
    return rng.uniform(0.0, W, size=N), rng.uniform(0.0, H, size=N)


def gaussian_params(N: int, C: int, H: int, W: int, seed: int, s_min_px: float = 0.5,
                    s_max_px: float = 4.0, dtype=np.float32) -> dict:
    """Pre-activation Gaussian parameters, structure of arrays:
    xy_raw [N,2], s_raw [N,2], theta [N], amp [N,C], phase [N,C], alpha_raw [N]."""
    rng = np.random.default_rng(seed)
    x, y = _draw_means(rng, N, H, W)
    lim = 1.0 - 1e-6
    xy_raw = np.stack([np.arctanh(np.clip(2.0 * x / W - 1.0, -lim, lim)),
                       np.arctanh(np.clip(2.0 * y / H - 1.0, -lim, lim))], axis=1)
    s_act = np.exp(rng.uniform(np.log(s_min_px), np.log(s_max_px), size=(N, 2)))
    s_raw = np.log(np.maximum(s_act - 0.1, 1e-6))
    theta = rng.uniform(0.0, np.pi, size=N)
    amp = rng.uniform(0.0, 1.0, size=(N, C))
    phase = rng.uniform(0.0, 2.0 * np.pi, size=(N, C))
    alpha_raw = np.full(N, -0.5)
    p = {"xy_raw": xy_raw, "s_raw": s_raw, "theta": theta, "amp": amp, "phase": phase,
         "alpha_raw": alpha_raw}
    return {k: np.ascontiguousarray(v.astype(dtype)) for k, v in p.items()}


def params_for(w: Workload, dtype=np.float32, seed: Optional[int] = None) -> dict:
    return gaussian_params(w.N, w.C, w.H, w.W, w.seed if seed is None else seed,
                           w.s_min_px, w.s_max_px, dtype)


def blob_targets(L: int, C: int, H: int, W: int, seed: int = SEED_TARGETS, blobs: int = 8,
                 dtype=np.float32) -> np.ndarray:
    """Smooth synthetic target intensities [L, C, H, W] in [0, 1]."""
    rng = np.random.default_rng(seed)
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    out = np.zeros((L, C, H, W), np.float64)
    for l in range(L):
        for c in range(C):
            img = np.zeros((H, W))
            for _ in range(blobs):
                cx, cy = rng.uniform(0, W), rng.uniform(0, H)
                sig = rng.uniform(8.0, 40.0)
                peak = rng.uniform(0.3, 1.0)
                img += peak * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2.0 * sig * sig))
            m = img.max()
            out[l, c] = img / m if m > 0 else img
    return out.astype(dtype)


def random_field(C: int, H: int, W: int, seed: int, dtype=np.complex64) -> np.ndarray:
    """Complex Gaussian random field [C, H, W] (for propagation-only tests)."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((C, H, W)) + 1j * rng.standard_normal((C, H, W))
    return f.astype(dtype)


def sample_indices(count: int, total: int, seed: int) -> np.ndarray:
    """Seeded sample of distinct indices in [0, total) (sorted)."""
    rng = np.random.default_rng(seed)
    count = min(count, total)
    return np.sort(rng.choice(total, size=count, replace=False)).astype(np.int64)


def planted_scene(N: int, C: int, H: int, W: int, seed: int, blobs: int = 8,
                  dtype=np.float32) -> dict:
    """Pre-activation parameters of a structured planted scene: gaussian_params draws with
    every phase zero and each channel's amplitude read from a smooth field (a sum of
    `blobs` isotropic Gaussian blobs, sigma U(H/24, H/6), peak U(0.3, 1), normalised to
    maximum 1) at the Gaussian's mean.  A random-phase scene would render as speckle; this
    one renders as an image-like intensity that the scene's own parameters reproduce."""
    p = gaussian_params(N, C, H, W, seed, dtype=np.float64)
    # the same mean draws gaussian_params started from (same seed, same first draws)
    x, y = _draw_means(np.random.default_rng(seed), N, H, W)
    rng = np.random.default_rng(seed ^ 0x5EED)
    amp = np.zeros((N, C))
    for c in range(C):
        for _ in range(blobs):
            cx, cy = rng.uniform(0, W), rng.uniform(0, H)
            sig = rng.uniform(H / 24.0, H / 6.0)
            amp[:, c] += rng.uniform(0.3, 1.0) * np.exp(-((x - cx) ** 2 + (y - cy) ** 2)
                                                        / (2.0 * sig * sig))
        m = amp[:, c].max()
        if m > 0:
            amp[:, c] /= m
    p["amp"] = amp
    p["phase"] = np.zeros((N, C))
    return {k: np.ascontiguousarray(v.astype(dtype)) for k, v in p.items()}


def depth_masks(L: int, H: int, W: int, seed: int, blobs: int = 6) -> np.ndarray:
    """Binary depth masks [L, H, W] uint8 for the reconstruction loss: a smooth synthetic
    depth map (sum of isotropic blobs, sigma U(H/8, H/3)) normalised to [0, 1) and
    quantised into L levels; mask l marks the pixels whose depth falls in level l (the
    paper's masks come from a depth estimator, which is not available here)."""
    rng = np.random.default_rng(seed)
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    depth = np.zeros((H, W))
    for _ in range(blobs):
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        sig = rng.uniform(H / 8.0, H / 3.0)
        depth += rng.uniform(0.2, 1.0) * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig * sig))
    lo, hi = depth.min(), depth.max()
    depth = (depth - lo) / (hi - lo + 1e-12) * (1.0 - 1e-9)
    q = np.minimum((depth * L).astype(np.int64), L - 1)
    return np.stack([(q == l).astype(np.uint8) for l in range(L)])
