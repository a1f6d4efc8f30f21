"""Pins of the oracle's loss, Adam and the composed forward/backward: closed forms,
finite differences through the whole chain, and torch.optim.Adam."""
import numpy as np
import pytest


def test_mse_closed_form_and_gradient(orc):
    rng = np.random.default_rng(0)
    L, C, H, W = 2, 2, 5, 6
    T = rng.uniform(0, 1, (L, C, H, W))
    loss0, _ = orc.mse_loss(np.zeros((L, C, H, W), complex), T)
    assert abs(loss0 - np.mean(T ** 2)) < 1e-15
    Ud = rng.standard_normal((L, C, H, W)) + 1j * rng.standard_normal((L, C, H, W))
    loss, g = orc.mse_loss(Ud, T)
    for idx in [(0, 0, 0, 0), (1, 1, 4, 5), (0, 1, 2, 3)]:
        for part in (1.0, 1j):
            h = 1e-6
            Up = Ud.copy(); Up[idx] += h * part
            Um = Ud.copy(); Um[idx] -= h * part
            fd = (orc.mse_loss(Up, T)[0] - orc.mse_loss(Um, T)[0]) / (2 * h)
            an = g[idx].real if part == 1.0 else g[idx].imag
            assert abs(fd - an) < 1e-7 * max(1, abs(an))


def test_psnr_closed_form(orc):
    L, C, H, W = 2, 1, 4, 4
    T = np.full((L, C, H, W), 0.5)
    Ud = np.sqrt(np.full((L, C, H, W), 0.6)).astype(complex)  # I = 0.6, error 0.1
    assert abs(orc.psnr(Ud, T) - 20.0) < 1e-9


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    import oracle as orc
    rng = np.random.default_rng(1)
    p = rng.standard_normal(7)
    m = np.zeros(7); v = np.zeros(7)
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.01)
    for t in range(1, 6):
        g = rng.standard_normal(7)
        orc.adam(p, g, m, v, 0.01, t)
        opt.zero_grad()
        tp.grad = torch.tensor(g)
        opt.step()
        assert np.abs(p - tp.detach().numpy()).max() < 1e-14


def test_adam_scalar_recurrence(orc):
    """First step moves every coordinate by lr * sign(g) (bias-corrected m/sqrt(v) = g/|g|)."""
    p = np.array([1.0, -2.0, 3.0]); g = np.array([0.5, -4.0, 1e-3])
    m = np.zeros(3); v = np.zeros(3)
    orc.adam(p, g, m, v, 0.1, 1)
    assert np.allclose(p, np.array([0.9, -1.9, 2.9]), atol=1e-6)


def test_full_chain_finite_differences(orc):
    """dL/dparams from raster -> BLASM -> MSE -> adjoint BLASM -> raster backward equals
    central differences of the forward loss (smooth mode, two planes, two colours)."""
    rng = np.random.default_rng(3)
    H, W, C, N = 12, 16, 2, 5
    lam, z, pitch = [638e-9, 450e-9], [0.0, 3e-3], 8e-6
    p = {"xy_raw": rng.uniform(-1, 1, (N, 2)), "s_raw": rng.uniform(0.2, 1.0, (N, 2)),
         "theta": rng.uniform(0, np.pi, N), "amp": rng.uniform(0.2, 1, (N, C)),
         "phase": rng.uniform(0, 2 * np.pi, (N, C)), "alpha_raw": rng.uniform(-1, 1, N)}
    T = rng.uniform(0, 0.3, (len(z), C, H, W))

    def loss(q):
        _, Ud = orc.forward(q, H, W, lam, pitch, z, cutoff=0.0)
        return orc.mse_loss(Ud, T)[0]

    out = orc.step(p, T, H, W, lam, pitch, z, cutoff=0.0)
    assert abs(out["loss"] - loss(p)) < 1e-15
    # central differences carry ~eps * loss / h of rounding noise: an absolute floor
    gmax = max(np.abs(g).max() for g in out["grads"].values())
    for key in p:
        for flat in range(min(p[key].size, 4)):
            idx = np.unravel_index(flat, p[key].shape)
            h = 1e-6 * max(1.0, abs(p[key][idx]))
            qp = {k: v.copy() for k, v in p.items()}; qp[key][idx] += h
            qm = {k: v.copy() for k, v in p.items()}; qm[key][idx] -= h
            fd = (loss(qp) - loss(qm)) / (2 * h)
            an = out["grads"][key][idx]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), abs(an)) + 1e-8 * gmax, (key, idx, fd, an)
