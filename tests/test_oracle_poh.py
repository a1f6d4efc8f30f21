"""Pins of the POH-conversion oracle (Sec. 3.3): the spectrum of the DPAC pattern of a
constant field (numpy's FFT, closed form), L_extract's reduction to twice the pinned
L_recon when both fields agree, its complex-L1 term for a constant difference, finite
differences of its gradients, of the phase gradient and of the whole conversion step."""
import numpy as np

import oracle
from oracle import poh_ref as pr


def test_dpac_printed_form_of_a_constant_field_is_a_checkerboard():
    a, th = 0.7, -1.2
    H, W = 6, 8
    Hf = np.full((1, H, W), a * np.exp(1j * th))
    out = pr.dpac(Hf, mode="printed")
    assert np.allclose(np.abs(out), 1.0)
    F = np.fft.fft2(out[0])
    n = H * W
    assert abs(F[0, 0] - n / 2 * (np.exp(1j * a) + np.exp(1j * th))) < 1e-12
    assert abs(F[H // 2, W // 2] - n / 2 * (np.exp(1j * a) - np.exp(1j * th))) < 1e-12
    rest = np.abs(F).copy()
    rest[0, 0] = rest[H // 2, W // 2] = 0.0
    assert rest.max() < 1e-12


def test_double_phase_pairs_average_to_the_normalised_field():
    """cos-addition: (exp(j(phi + a)) + exp(j(phi - a))) / 2 = cos(a) exp(j phi), so on a
    field constant over horizontal pixel pairs every pair of the coded field averages to
    (|H| / max|H|) exp(j arg H)."""
    rng = np.random.default_rng(9)
    C, H, W = 2, 4, 6
    half = rng.uniform(0.1, 2.0, size=(C, H, W // 2)) * np.exp(1j * rng.uniform(-3, 3, size=(C, H, W // 2)))
    Hf = np.repeat(half, 2, axis=2)
    out = pr.dpac(Hf)
    assert np.allclose(np.abs(out), 1.0)
    pair_mean = 0.5 * (out[:, :, 0::2] + out[:, :, 1::2])
    amax = np.abs(half).reshape(C, -1).max(axis=1)[:, None, None]
    assert np.abs(pair_mean - half / amax).max() < 1e-12


def _fields(seed, L=2, C=2, H=4, W=5):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((L, C, H, W)) + 1j * rng.standard_normal((L, C, H, W))
    R = rng.standard_normal((L, C, H, W)) + 1j * rng.standard_normal((L, C, H, W))
    T = rng.uniform(0.0, 1.0, size=(L, C, H, W))
    M = (rng.uniform(size=(L, H, W)) < 0.5).astype(np.uint8)
    return U, R, T, M


def test_extract_loss_with_equal_fields_is_twice_recon():
    U, _, T, M = _fields(1)
    loss, dU, dR = pr.extract_loss(U, U, T, M)
    r, g = oracle.recon_loss(U, T, M)
    L = U.shape[0]
    assert abs(loss - 2 * L * r) < 1e-12 * loss
    assert np.abs(dU - L * g).max() < 1e-12 and np.abs(dR - L * g).max() < 1e-12


def test_extract_field_term_constant_difference():
    U, _, T, M = _fields(2)
    d = 0.3 - 0.45j
    R = U - d
    l0 = pr.extract_loss(U, R, T, M, lambda_comp=0.0, lambda_field=0.0)[0]
    l1 = pr.extract_loss(U, R, T, M, lambda_comp=0.0, lambda_field=0.01)[0]
    L = U.shape[0]
    assert abs((l1 - l0) - 0.01 * L * (abs(d.real) + abs(d.imag))) < 1e-14


def test_extract_loss_gradients_finite_differences():
    U, R, T, M = _fields(3, L=1, C=1, H=3, W=4)
    loss, dU, dR = pr.extract_loss(U, R, T, M, lambda_comp=0.3, lambda_field=0.05)
    h = 1e-7
    for which, grad in ((0, dU), (1, dR)):
        for idx in [(0, 0, 0, 0), (0, 0, 1, 2), (0, 0, 2, 3)]:
            for comp, g in ((1.0, grad[idx].real), (1j, grad[idx].imag)):
                a = [U.copy(), R.copy()]
                b = [U.copy(), R.copy()]
                a[which][idx] += h * comp
                b[which][idx] -= h * comp
                fd = (pr.extract_loss(a[0], a[1], T, M, 0.3, 0.05)[0] -
                      pr.extract_loss(b[0], b[1], T, M, 0.3, 0.05)[0]) / (2 * h)
                assert abs(fd - g) < 1e-6 * max(1.0, abs(g))


def test_phase_gradient_finite_differences():
    rng = np.random.default_rng(4)
    phi = rng.uniform(-3, 3, size=(2, 3, 4))
    G = rng.standard_normal(phi.shape) + 1j * rng.standard_normal(phi.shape)

    def f(p):  # a linear functional of H = exp(j p): sum Re(conj(G) H), so dL/dH = G
        return float(np.sum((np.conj(G) * pr.poh_field(p)).real))

    d = pr.phase_grad(phi, G)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 3), (0, 1, 2)]:
        a, b = phi.copy(), phi.copy()
        a[idx] += h
        b[idx] -= h
        assert abs((f(a) - f(b)) / (2 * h) - d[idx]) < 1e-8


def test_poh_step_finite_differences():
    from paper_2511_15022_gb300 import inputs
    w = inputs.custom(12, 10, 6, wavelengths_m=(520e-9,), z_m=(0.0, 3e-3), seed=5,
                      cutoff=0.0)
    p = {k: v.astype(np.float64) for k, v in inputs.params_for(w).items()}
    rng = np.random.default_rng(6)
    phi = rng.uniform(-np.pi, np.pi, size=(w.C, w.H, w.W))
    T = inputs.blob_targets(w.L, w.C, w.H, w.W).astype(np.float64)
    M = inputs.depth_masks(w.L, w.H, w.W, seed=7)
    args = (w.H, w.W, w.wavelengths_m, w.pitch_m, w.z_m, w.pad, 0.0, M)
    out = pr.poh_step(p, phi, T, *args)
    h = 1e-6
    for idx in [(0, 0, 0), (0, 5, 7), (0, 11, 9)]:
        a, b = phi.copy(), phi.copy()
        a[idx] += h
        b[idx] -= h
        fd = (pr.poh_step(p, a, T, *args)["loss"] - pr.poh_step(p, b, T, *args)["loss"]) / (2 * h)
        assert abs(fd - out["dphi"][idx]) < 1e-6 * max(1e-3, abs(fd))
    for k, idx in (("amp", (2, 0)), ("xy_raw", (1, 0)), ("phase", (4, 0))):
        a = {q: v.copy() for q, v in p.items()}
        b = {q: v.copy() for q, v in p.items()}
        a[k][idx] += h
        b[k][idx] -= h
        fd = (pr.poh_step(a, phi, T, *args)["loss"] - pr.poh_step(b, phi, T, *args)["loss"]) / (2 * h)
        assert abs(fd - out["grads"][k][idx]) < 1e-5 * max(1e-3, abs(fd)), k
