"""Helpers shared by the GPU parity tests (marshalling and error measures only)."""
import numpy as np


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def to_dev(p_np: dict, dev):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v.astype(np.float32))).to(dev)
            for k, v in p_np.items()}


def to64(p_np: dict) -> dict:
    return {k: np.asarray(v, dtype=np.float64) for k, v in p_np.items()}


def c64(t) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.complex128)
