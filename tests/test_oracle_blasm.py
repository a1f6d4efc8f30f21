"""Pins of the oracle's band-limited angular spectrum method (Algorithm 3; Sec. 2 transfer
function) against physics and closed forms: z = 0 identity, |H| = 1 in band (Parseval),
the main-text form exp(j 2 pi d sqrt(1/lambda^2 - r^2)), H(d1) H(d2) = H(d1 + d2),
H(-d) = conj H(d), the exact band-limit mask count, and the adjoint identity of the
backward (Suppl. BLASM backward)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_zero_distance_is_identity(orc):
    rng = np.random.default_rng(0)
    U0 = rng.standard_normal((2, 12, 18)) + 1j * rng.standard_normal((2, 12, 18))
    Ud = orc.blasm_fwd(U0, [638e-9, 450e-9], 8e-6, [0.0])
    assert np.abs(Ud[0] - U0).max() < 1e-12


def test_transfer_matches_main_text_form(orc):
    """Supplementary k_z = sqrt(k^2 - (2 pi)^2 r^2) equals the main-text
    2 pi sqrt(1/lambda^2 - r^2); in band |H| = 1."""
    ny, nx, lam, pitch, d = 40, 60, 520e-9, 8e-6, 7e-3
    Hf = orc.blasm_transfer(ny, nx, lam, pitch, d)
    fx = np.fft.fftfreq(nx, d=pitch)
    fy = np.fft.fftfreq(ny, d=pitch)
    r2 = fx[None, :] ** 2 + fy[:, None] ** 2
    ref = np.exp(1j * 2 * np.pi * d * np.sqrt(1 / lam ** 2 - r2))
    band = np.abs(Hf) > 0  # the rectangular band limit is active on this small grid
    assert 0.3 * Hf.size < band.sum() < Hf.size
    assert np.abs(Hf - ref)[band].max() < 1e-9
    assert np.abs(np.abs(Hf[band]) - 1).max() < 1e-12


def test_parseval_unmasked(orc):
    """Unmasked propagation preserves energy on the padded grid."""
    rng = np.random.default_rng(1)
    ny, nx = 32, 48
    P = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    Hf = orc.blasm_transfer(ny, nx, 638e-9, 8e-6, 1e-3)  # d small enough: no bin masked
    assert np.all(np.abs(Hf) > 0)
    out = orc.fft2d(Hf * orc.fft2d(P), inverse=True) / P.size
    assert abs(np.vdot(out, out).real - np.vdot(P, P).real) < 1e-10 * np.vdot(P, P).real


def test_round_trip_and_conjugate_symmetry(orc):
    ny, nx = 30, 40
    for d in [1e-3, 12e-3, 50e-3]:
        Hp = orc.blasm_transfer(ny, nx, 520e-9, 8e-6, d)
        Hm = orc.blasm_transfer(ny, nx, 520e-9, 8e-6, -d)
        assert np.abs(Hm - np.conj(Hp)).max() < 1e-12
        band = np.abs(Hp) > 0
        assert np.abs((Hp * Hm)[band] - 1).max() < 1e-12
    # propagate z then -z on the padded grid (no intermediate crop): identity in band
    rng = np.random.default_rng(2)
    P = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    Hp = orc.blasm_transfer(ny, nx, 520e-9, 8e-6, 1e-3)
    Hm = orc.blasm_transfer(ny, nx, 520e-9, 8e-6, -1e-3)
    assert np.all(np.abs(Hp) > 0)
    fwd = orc.fft2d(Hp * orc.fft2d(P), inverse=True) / P.size
    back = orc.fft2d(Hm * orc.fft2d(fwd), inverse=True) / P.size
    assert np.abs(back - P).max() < 1e-12


def test_composition(orc):
    ny, nx = 24, 36
    H1 = orc.blasm_transfer(ny, nx, 450e-9, 8e-6, 1e-3)
    H2 = orc.blasm_transfer(ny, nx, 450e-9, 8e-6, 1.5e-3)
    H12 = orc.blasm_transfer(ny, nx, 450e-9, 8e-6, 2.5e-3)
    assert np.all(np.abs(H12) > 0)  # band limit inactive at these distances
    assert np.abs(H1 * H2 - H12).max() < 1e-9


def test_plane_wave_eigenmode(orc):
    """A plane wave on the (periodic) padded grid is an eigenmode: propagation multiplies
    it by H at its frequency."""
    ny, nx, pitch, lam, d = 16, 20, 8e-6, 638e-9, 0.5e-3
    kx, ky = 3, 13  # ky = 13 is the negative frequency -3 on a 16-point grid
    y, x = np.mgrid[0:ny, 0:nx]
    wave = np.exp(2j * np.pi * (kx * x / nx + ky * y / ny))
    Hf = orc.blasm_transfer(ny, nx, lam, pitch, d)
    out = orc.fft2d(Hf * orc.fft2d(wave), inverse=True) / wave.size
    fx, fy = kx / (nx * pitch), (ky - ny) / (ny * pitch)
    h = np.exp(1j * 2 * np.pi * d * np.sqrt(1 / lam ** 2 - fx ** 2 - fy ** 2))
    assert np.abs(out - h * wave).max() < 1e-11


def test_band_limit_mask_count_golden(orc):
    """64x64 at 8 um, 520 nm, d = 50 mm, padded to 128x128: f_max = 1/(lambda
    sqrt((2d/L)^2 + 1)) with L = 1.024 mm admits |s| <= 20 per axis -> 41 x 41 bins."""
    with open(os.path.join(GOLDEN, "bandlimit_mask_128x128_520nm_50mm.txt")) as f:
        fields = dict(line.split("=", 1) for line in f.read().split("\n")
                      if "=" in line and not line.startswith("#"))
    n = int(fields["n"])
    Hf = orc.blasm_transfer(n, n, float(fields["lambda_m"]), float(fields["pitch_m"]),
                            float(fields["d_m"]))
    mask = np.abs(Hf) > 0
    assert mask.sum() == int(fields["count"])
    s = np.fft.fftfreq(n, d=1.0 / n).astype(int)
    kept = s[mask.any(axis=0)]
    assert kept.max() == int(fields["max_index"]) and kept.min() == -int(fields["max_index"])


def test_aperture_radius(orc):
    """Algorithm 3's optional circular aperture removes bins at index distance >= a from
    the centre N/2 - 0.5 of the centred layout."""
    n = 32
    Hf = orc.blasm_transfer(n, n, 520e-9, 8e-6, 1e-3, aperture=6.0)
    s = np.fft.fftfreq(n, d=1.0 / n)
    ax = s[None, :] + 0.5
    ay = s[:, None] + 0.5
    inside = ax ** 2 + ay ** 2 < 36.0
    assert np.array_equal(np.abs(Hf) > 0, inside)


def test_backward_is_adjoint(orc):
    """Re <A x, y> = Re <x, A^H y> for the multi-plane forward/backward pair."""
    rng = np.random.default_rng(3)
    C, H, W, L = 2, 10, 14, 3
    lam, z = [638e-9, 450e-9], [0.0, 2e-3, 30e-3]
    x = rng.standard_normal((C, H, W)) + 1j * rng.standard_normal((C, H, W))
    y = rng.standard_normal((L, C, H, W)) + 1j * rng.standard_normal((L, C, H, W))
    Ax = orc.blasm_fwd(x, lam, 8e-6, z)
    Ahy = orc.blasm_bwd(y, lam, 8e-6, z)
    lhs = np.vdot(Ax, y).real
    rhs = np.vdot(x, Ahy).real
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))


def test_odd_sizes_pad_offsets(orc):
    """Odd image sizes: the centred window of the 2x padded grid starts at (N - n) // 2;
    at z = 0 the crop returns the input exactly."""
    rng = np.random.default_rng(4)
    U0 = rng.standard_normal((1, 7, 9)) + 1j * rng.standard_normal((1, 7, 9))
    assert np.abs(orc.blasm_fwd(U0, [520e-9], 8e-6, [0.0])[0] - U0).max() < 1e-12
