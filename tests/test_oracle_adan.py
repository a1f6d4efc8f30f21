"""Pins of the oracle's Adan step (Sec. 4 trains with Adan): with beta2 = 0 it is Adam
exactly (the Adam oracle is pinned to torch.optim.Adam), a constant gradient gives the
closed-form trajectory p_t = p_0 - t lr g / (|g| + eps), the update is invariant to the
gradient scale when eps = 0, and weight decay divides by 1 + lr wd."""
import numpy as np

import oracle


def _run_adan(grads, lr, **kw):
    p = np.array([0.3, -1.1, 2.0, 0.0])
    m, v, n, gp = (np.zeros_like(p) for _ in range(4))
    traj = []
    for t, g in enumerate(grads, start=1):
        oracle.adan(p, g, m, v, n, gp, lr, t, **kw)
        traj.append(p.copy())
    return np.array(traj)


def test_adan_with_beta2_zero_is_adam():
    rng = np.random.default_rng(3)
    grads = rng.standard_normal((12, 4))
    a = _run_adan(grads, 0.01, beta1=0.9, beta2=0.0, beta3=0.999)
    p = np.array([0.3, -1.1, 2.0, 0.0])
    m, v = np.zeros_like(p), np.zeros_like(p)
    for t, g in enumerate(grads, start=1):
        oracle.adam(p, g, m, v, 0.01, t, beta1=0.9, beta2=0.999)
        assert np.abs(a[t - 1] - p).max() < 1e-14


def test_adan_constant_gradient_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 3.0])
    traj = _run_adan([g] * 20, 0.05, eps=1e-8)
    p0 = np.array([0.3, -1.1, 2.0, 0.0])
    for t in (1, 5, 20):
        want = p0 - t * 0.05 * g / (np.abs(g) + 1e-8)
        assert np.abs(traj[t - 1] - want).max() < 1e-12


def test_adan_is_invariant_to_the_gradient_scale():
    rng = np.random.default_rng(4)
    grads = rng.standard_normal((10, 4))
    a = _run_adan(grads, 0.02, eps=0.0)
    b = _run_adan(grads * 37.0, 0.02, eps=0.0)
    assert np.abs(a - b).max() < 1e-12


def test_adan_weight_decay_divides():
    g = np.zeros(4)
    traj = _run_adan([g, g], 0.1, weight_decay=0.5, eps=1.0)
    p0 = np.array([0.3, -1.1, 2.0, 0.0])
    assert np.abs(traj[1] - p0 / (1 + 0.05) ** 2).max() < 1e-14
