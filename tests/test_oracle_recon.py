"""Pins of the oracle's reconstruction loss L_recon (Sec. 3.2): its three terms are the
intensity MSE of transformed inputs -- |U sqrt(M)|^2 = I M against I^ M and |U sqrt(I^)|^2 =
I I^ against I^ I^ -- so the pinned MSE oracle checks each of them; plus finite
differences of its gradient, a closed form and the no-mask case."""
import numpy as np

import oracle


def _case(seed, L=2, C=3, H=5, W=7):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((L, C, H, W)) + 1j * rng.standard_normal((L, C, H, W))
    T = rng.uniform(0.0, 1.5, size=(L, C, H, W))
    M = (rng.uniform(size=(L, H, W)) < 0.4).astype(np.uint8)
    return U, T, M


def test_recon_is_the_sum_of_three_intensity_mses():
    U, T, M = _case(1)
    loss, dU = oracle.recon_loss(U, T, M)
    Mc = M[:, None, :, :].astype(np.float64)  # shared by the colour channels
    l1, g1 = oracle.mse_loss(U, T)
    l2, g2 = oracle.mse_loss(U * np.sqrt(Mc), T * Mc)
    l3, g3 = oracle.mse_loss(U * np.sqrt(T), T * T)
    assert abs(loss - (l1 + l2 + l3)) < 1e-12 * max(1.0, loss)
    # chain rule through the real factors sqrt(M) and sqrt(I^)
    want = g1 + np.sqrt(Mc) * g2 + np.sqrt(T) * g3
    assert np.abs(dU - want).max() < 1e-12 * max(1.0, np.abs(want).max())


def test_recon_gradient_finite_differences():
    U, T, M = _case(2, L=1, C=2, H=3, W=4)
    _, dU = oracle.recon_loss(U, T, M)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 2, 3), (0, 1, 1, 2), (0, 0, 2, 1)]:
        for comp, g in ((1.0, dU[idx].real), (1j, dU[idx].imag)):
            Up, Um = U.copy(), U.copy()
            Up[idx] += h * comp
            Um[idx] -= h * comp
            fd = (oracle.recon_loss(Up, T, M)[0] - oracle.recon_loss(Um, T, M)[0]) / (2 * h)
            assert abs(fd - g) < 1e-7 * max(1.0, abs(g))


def test_recon_closed_form_constant_fields():
    L, C, H, W = 2, 1, 4, 4
    u, t = 0.8 + 0.3j, 0.25
    U = np.full((L, C, H, W), u)
    T = np.full((L, C, H, W), t)
    M = np.ones((L, H, W), np.uint8)
    I0 = abs(u) ** 2
    loss, _ = oracle.recon_loss(U, T, M)
    assert abs(loss - (I0 - t) ** 2 * (2.0 + t * t)) < 1e-14


def test_recon_without_mask_and_target_is_mse():
    U, T, M = _case(3)
    zeroT = np.zeros_like(T)
    assert abs(oracle.recon_loss(U, zeroT, None)[0] - oracle.mse_loss(U, zeroT)[0]) < 1e-14
    a = oracle.recon_loss(U, T, None)
    b = oracle.recon_loss(U, T, np.zeros_like(M))
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
