"""Pins of the oracle's own transforms (oracle/fourier.py) against brute force and identities."""
import cmath
import itertools

import numpy as np
import pytest

from oracle import fourier


def brute_force_coeffs(f):
    """Fourier coefficients by the definition, pure-Python loops (tiny grids only)."""
    n3, n2, n1 = f.shape
    m = n1 * n2 * n3
    out = np.zeros(f.shape, dtype=complex)
    for k3, k2, k1 in itertools.product(range(n3), range(n2), range(n1)):
        s = 0j
        for a3, a2, a1 in itertools.product(range(n3), range(n2), range(n1)):
            ph = -2j * cmath.pi * (k1 * a1 / n1 + k2 * a2 / n2 + k3 * a3 / n3)
            s += f[a3, a2, a1] * cmath.exp(ph)
        out[k3, k2, k1] = s / m
    return out


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 3, 3), (6, 6, 6), (4, 3, 2), (2, 8, 6)])
def test_forward_matches_brute_force(shape):
    rng = np.random.default_rng(1)
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    np.testing.assert_allclose(fourier.forward(f), brute_force_coeffs(f), rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 12, 4), (9, 16, 24)])
def test_inverse_roundtrip_and_parseval(shape):
    rng = np.random.default_rng(2)
    f = rng.standard_normal((2,) + shape)
    fh = fourier.forward(f)
    np.testing.assert_allclose(fourier.inverse(fh).real, f, atol=1e-12)
    # Parseval for the Fourier-series convention: mean |f|^2 = sum |f_hat|^2
    np.testing.assert_allclose(np.mean(f ** 2, axis=(1, 2, 3)),
                               np.sum(np.abs(fh) ** 2, axis=(1, 2, 3)), rtol=1e-12)


@pytest.mark.parametrize("shape", [(16, 8, 32), (12, 6, 18)])
def test_against_numpy_fft(shape):
    """numpy.fft is an outside cross-check only; the oracle never calls it."""
    rng = np.random.default_rng(3)
    f = rng.standard_normal(shape)
    np.testing.assert_allclose(fourier.forward(f), np.fft.fftn(f) / f.size, atol=1e-14)


def test_frequencies_and_nyquist():
    assert list(fourier.frequencies(4)) == [0, 1, -2, -1]
    assert list(fourier.frequencies(3)) == [0, 1, -1]
    assert list(fourier.frequencies(6)) == [0, 1, 2, -3, -2, -1]
    m = fourier.nyquist_mask((4, 3, 2))
    assert m.shape == (2, 3, 4)
    assert m[:, :, 2].all() and m[1].all() and not m[0, :, :2].any()


def test_plane_wave_derivative_sign():
    """f = cos(xi . y) has f_hat = 1/2 at +-k: the e^{+i xi y} convention of the paper."""
    n = 8
    y = np.arange(n)
    f = np.cos(2 * np.pi * 1 * y / n)[None, None, :] * np.ones((n, n, 1))
    fh = fourier.forward(f)
    assert abs(fh[0, 0, 1] - 0.5) < 1e-14 and abs(fh[0, 0, n - 1] - 0.5) < 1e-14
