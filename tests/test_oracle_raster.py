"""Pins of the oracle rasteriser (Algorithm 2, Sec. 3.1) against facts that do not come
from the oracle itself: the closed-form Fourier transform of a 2D Gaussian, Poisson
summation, geometric symmetries, linearity, the 0.99 / 1/255 rules of Algorithm 2 and
finite differences of the forward for the analytic backward."""
import numpy as np
import pytest


def one_gaussian(mx, my, sx, sy, theta, amp, phase, alpha_raw, W, H):
    """Pre-activation parameters reproducing the given activated mean and scales."""
    xr = np.arctanh(2.0 * mx / W - 1.0)
    yr = np.arctanh(2.0 * my / H - 1.0)
    C = len(amp)
    return {
        "xy_raw": np.array([[xr, yr]]),
        "s_raw": np.log(np.array([[sx - 0.1, sy - 0.1]])),
        "theta": np.array([theta]),
        "amp": np.array([amp], float).reshape(1, C),
        "phase": np.array([phase], float).reshape(1, C),
        "alpha_raw": np.array([alpha_raw]),
    }


def cov_matrix(sx, sy, theta):
    """Sigma = R diag(s^2) R^T + 0.1 I as a matrix product (Suppl. 2D covariance)."""
    R = np.array([[np.cos(theta), -np.sin(theta)], [np.sin(theta), np.cos(theta)]])
    return R @ np.diag([sx * sx, sy * sy]) @ R.T + 0.1 * np.eye(2)


@pytest.mark.parametrize("theta", [0.0, 0.4, 1.3, 2.9])
def test_closed_form_fourier_transform(orc, theta):
    """DFT of one rendered Gaussian equals 2 pi sqrt(det S) exp(-2 pi^2 f^T S f)
    exp(-2 pi i f.x) times alpha c exp(i phi) at low frequencies (smooth mode)."""
    H = W = 64
    mx, my, sx, sy = 31.3, 32.6, 3.5, 1.6
    amp, ph, ar = 0.7, 0.9, -0.5
    p = one_gaussian(mx, my, sx, sy, theta, [amp], [ph], ar, W, H)
    U = orc.raster_fwd(p, H, W, cutoff=0.0)[0]
    F = np.fft.fft2(U)
    S = cov_matrix(sx, sy, theta)
    alpha = 1.0 / (1.0 + np.exp(-ar))
    k = np.fft.fftfreq(W)  # cycles per pixel
    worst = 0.0
    for ky in range(H):
        for kx in range(W):
            f = np.array([k[kx], k[ky]])
            if np.abs(f).max() > 0.2:
                continue
            ref = (alpha * amp * np.exp(1j * ph) * 2 * np.pi * np.sqrt(np.linalg.det(S))
                   * np.exp(-2 * np.pi ** 2 * f @ S @ f)
                   * np.exp(-2j * np.pi * (f[0] * mx + f[1] * my)))
            worst = max(worst, abs(F[ky, kx] - ref))
    assert worst < 1e-9


def test_poisson_summation_mass(orc):
    """sum_p G(p) = 2 pi sqrt(det Sigma) for a Gaussian far from the edges."""
    H, W = 48, 56
    for sx, sy, th in [(1.5, 1.5, 0.0), (2.0, 4.0, 0.7), (3.0, 1.7, 2.2)]:
        p = one_gaussian(27.4, 23.9, sx, sy, th, [1.0], [0.0], -0.5, W, H)
        U = orc.raster_fwd(p, H, W, cutoff=0.0)[0]
        alpha = 1.0 / (1.0 + np.exp(0.5))
        mass = U.sum().real / alpha
        ref = 2 * np.pi * np.sqrt(np.linalg.det(cov_matrix(sx, sy, th)))
        assert abs(mass - ref) < 1e-9 * ref


def test_peak_value_and_alpha_cap(orc):
    """At the mean pixel G = 1: the value is alpha c exp(i phi), and alpha is capped at 0.99
    (Algorithm 2)."""
    H = W = 32
    p = one_gaussian(10.0, 12.0, 2.0, 3.0, 0.3, [0.5], [1.1], -0.5, W, H)
    U = orc.raster_fwd(p, H, W)[0]
    alpha = 1.0 / (1.0 + np.exp(0.5))
    assert abs(U[12, 10] - alpha * 0.5 * np.exp(1.1j)) < 1e-12
    p = one_gaussian(10.0, 12.0, 2.0, 3.0, 0.3, [0.5], [1.1], 8.0, W, H)
    U = orc.raster_fwd(p, H, W)[0]
    assert abs(U[12, 10] - 0.99 * 0.5 * np.exp(1.1j)) < 1e-12


def test_cutoff_rule(orc):
    """With t = 1/255 a single Gaussian contributes exactly where alpha G >= t: the cut
    field equals the smooth field there and is zero elsewhere."""
    H, W = 40, 40
    p = one_gaussian(19.3, 20.8, 2.5, 1.2, 0.8, [1.0], [0.0], -0.5, W, H)
    Us = orc.raster_fwd(p, H, W, cutoff=0.0)[0]
    Uc = orc.raster_fwd(p, H, W, cutoff=1.0 / 255.0)[0]
    keep = np.abs(Us) >= 1.0 / 255.0  # amp = 1, phase = 0: |U| = alpha G
    assert np.array_equal(Uc[keep], Us[keep])
    assert np.all(Uc[~keep] == 0)
    assert 10 < keep.sum() < H * W


def test_symmetries(orc):
    """theta -> theta + pi and (sx, sy, theta) -> (sy, sx, theta + pi/2) leave the field
    unchanged; a common phase shift rotates it; amplitude scales it."""
    rng = np.random.default_rng(5)
    H, W, C, N = 24, 32, 2, 12
    p = {"xy_raw": rng.uniform(-1, 1, (N, 2)), "s_raw": rng.uniform(0, 1.2, (N, 2)),
         "theta": rng.uniform(0, np.pi, N), "amp": rng.uniform(0, 1, (N, C)),
         "phase": rng.uniform(0, 2 * np.pi, (N, C)), "alpha_raw": rng.uniform(-1, 1, N)}
    U = orc.raster_fwd(p, H, W, cutoff=0.0)
    q = dict(p, theta=p["theta"] + np.pi)
    assert np.abs(orc.raster_fwd(q, H, W, cutoff=0.0) - U).max() < 1e-12
    q = dict(p, s_raw=p["s_raw"][:, ::-1].copy(), theta=p["theta"] + np.pi / 2)
    assert np.abs(orc.raster_fwd(q, H, W, cutoff=0.0) - U).max() < 1e-12
    q = dict(p, phase=p["phase"] + 0.7)
    assert np.abs(orc.raster_fwd(q, H, W, cutoff=0.0) - U * np.exp(0.7j)).max() < 1e-12
    q = dict(p, amp=p["amp"] * 2.5)
    assert np.abs(orc.raster_fwd(q, H, W, cutoff=0.0) - 2.5 * U).max() < 1e-12
    # superposition: the field of a union of Gaussian sets is the sum of the fields
    a = {k: v[:5] for k, v in p.items()}
    b = {k: v[5:] for k, v in p.items()}
    Ua = orc.raster_fwd(a, H, W, cutoff=1 / 255)
    Ub = orc.raster_fwd(b, H, W, cutoff=1 / 255)
    assert np.abs(Ua + Ub - orc.raster_fwd(p, H, W, cutoff=1 / 255)).max() < 1e-12


def test_pixel_subset_matches_full(orc):
    rng = np.random.default_rng(9)
    H, W, C, N = 20, 28, 3, 30
    p = {"xy_raw": rng.uniform(-1.5, 1.5, (N, 2)), "s_raw": rng.uniform(-0.5, 1.5, (N, 2)),
         "theta": rng.uniform(0, np.pi, N), "amp": rng.uniform(0, 1, (N, C)),
         "phase": rng.uniform(0, 2 * np.pi, (N, C)), "alpha_raw": rng.uniform(-1, 3, N)}
    U = orc.raster_fwd(p, H, W)
    idx = np.array([0, 5, 77, 300, H * W - 1])
    Us = orc.raster_fwd(p, H, W, pix_idx=idx)
    assert np.array_equal(Us, U.reshape(C, -1)[:, idx])


def _rand_params(rng, N, C, spread=1.2, ar=(-1.0, 1.0)):
    return {"xy_raw": rng.uniform(-spread, spread, (N, 2)), "s_raw": rng.uniform(0.2, 1.3, (N, 2)),
            "theta": rng.uniform(0, np.pi, N), "amp": rng.uniform(0.1, 1, (N, C)),
            "phase": rng.uniform(0, 2 * np.pi, (N, C)), "alpha_raw": rng.uniform(*ar, N)}


def _fd_check(orc, p, H, W, C, cutoff, rel_tol):
    rng = np.random.default_rng(11)
    dU = rng.standard_normal((C, H, W)) + 1j * rng.standard_normal((C, H, W))

    def loss(q):
        U = orc.raster_fwd(q, H, W, cutoff=cutoff)
        return float(np.sum(dU.real * U.real + dU.imag * U.imag))

    g = orc.raster_bwd(p, H, W, dU, cutoff=cutoff)
    worst = 0.0
    for key in ("xy_raw", "s_raw", "theta", "amp", "phase", "alpha_raw"):
        arr = p[key]
        for flat in range(min(arr.size, 6)):
            idx = np.unravel_index(flat, arr.shape)
            h = 1e-6 * max(1.0, abs(arr[idx]))
            qp = {k: v.copy() for k, v in p.items()}
            qm = {k: v.copy() for k, v in p.items()}
            qp[key][idx] += h
            qm[key][idx] -= h
            fd = (loss(qp) - loss(qm)) / (2 * h)
            an = g[key][idx]
            err = abs(fd - an) / max(1e-6, abs(fd), abs(an))
            worst = max(worst, err)
            assert err < rel_tol, (key, idx, fd, an)
    return worst


def test_backward_finite_differences_smooth(orc):
    """Analytic backward (Suppl. gradient items 1-6 + the exact inverse-covariance
    derivative) against central differences of the forward, smooth mode."""
    rng = np.random.default_rng(1)
    H, W, C, N = 18, 22, 2, 6
    p = _rand_params(rng, N, C)
    _fd_check(orc, p, H, W, C, 0.0, 1e-6)


def test_backward_finite_differences_alpha_cap(orc):
    """Large opacity: pixels near the mean are capped at 0.99 and pass gradient only to
    amplitude and phase."""
    rng = np.random.default_rng(2)
    H, W, C, N = 18, 22, 1, 5
    p = _rand_params(rng, N, C, ar=(4.0, 6.0))
    p["xy_raw"] += 0.0123  # keep pixel centres off the cap boundary
    _fd_check(orc, p, H, W, C, 0.0, 1e-5)


def test_backward_subset_matches_full(orc):
    rng = np.random.default_rng(4)
    H, W, C, N = 16, 16, 2, 9
    p = _rand_params(rng, N, C)
    dU = rng.standard_normal((C, H, W)) + 1j * rng.standard_normal((C, H, W))
    g = orc.raster_bwd(p, H, W, dU)
    idx = np.array([1, 4, 8])
    gs = orc.raster_bwd(p, H, W, dU, g_idx=idx)
    for k in g:
        assert np.array_equal(gs[k], g[k][idx])


def test_backward_adjoint_identity(orc):
    """For the amplitude/phase directions the raster is linear in c exp(i phi):
    <dU, U(p + h e)> - <dU, U(p)> equals h * gradient exactly for amplitude."""
    rng = np.random.default_rng(6)
    H, W, C, N = 14, 14, 2, 4
    p = _rand_params(rng, N, C)
    dU = rng.standard_normal((C, H, W)) + 1j * rng.standard_normal((C, H, W))
    g = orc.raster_bwd(p, H, W, dU, cutoff=1 / 255)
    U0 = orc.raster_fwd(p, H, W, cutoff=1 / 255)
    q = {k: v.copy() for k, v in p.items()}
    q["amp"][2, 1] += 1.0
    U1 = orc.raster_fwd(q, H, W, cutoff=1 / 255)
    d = np.sum(dU.real * (U1 - U0).real + dU.imag * (U1 - U0).imag)
    assert abs(d - g["amp"][2, 1]) < 1e-12 * max(1, abs(d))
