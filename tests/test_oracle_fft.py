"""Pins of the oracle's textbook FFT: direct DFT, numpy.fft, impulse/constant pairs,
Parseval and round trips (forward exp(-2 pi i k n / N), unnormalised)."""
import numpy as np
import pytest

SIZES = [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 15, 16, 25, 27, 30, 45, 48, 60, 64, 98, 120]


@pytest.mark.parametrize("n", SIZES)
def test_fft_matches_direct_dft_and_numpy(orc, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = orc.fft1d(x)
    Xd = orc.dft1d(x)
    scale = max(1.0, np.abs(Xd).max())
    assert np.abs(X - Xd).max() / scale < 1e-12
    assert np.abs(X - np.fft.fft(x)).max() / scale < 1e-12
    xi = orc.fft1d(x, inverse=True)
    assert np.abs(xi - np.fft.ifft(x) * n).max() / scale < 1e-12


@pytest.mark.parametrize("n", [8, 15, 60])
def test_impulse_and_constant(orc, n):
    d = np.zeros(n, complex)
    d[0] = 1.0
    assert np.allclose(orc.fft1d(d), np.ones(n), atol=1e-14)
    c = np.ones(n, complex)
    e = np.zeros(n, complex)
    e[0] = n
    assert np.allclose(orc.fft1d(c), e, atol=1e-12)
    # shifted impulse -> pure phase ramp exp(-2 pi i k m / n)
    m = 3 % n
    s = np.zeros(n, complex)
    s[m] = 1.0
    k = np.arange(n)
    assert np.allclose(orc.fft1d(s), np.exp(-2j * np.pi * k * m / n), atol=1e-13)


@pytest.mark.parametrize("n", [12, 30, 64, 90])
def test_parseval_and_round_trip(orc, n):
    rng = np.random.default_rng(7 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = orc.fft1d(x)
    assert abs(np.vdot(X, X).real - n * np.vdot(x, x).real) < 1e-10 * n * np.vdot(x, x).real
    back = orc.fft1d(X, inverse=True) / n
    assert np.abs(back - x).max() < 1e-13


def test_fft2d_matches_numpy(orc):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((12, 20)) + 1j * rng.standard_normal((12, 20))
    X = orc.fft2d(x)
    assert np.abs(X - np.fft.fft2(x)).max() < 1e-11
    assert np.abs(orc.fft2d(X, inverse=True) / x.size - x).max() < 1e-13
