"""Oracle Fourier transforms (test infrastructure; see ``oracle/__init__``).

Convention (Sec. 2, periodic Lippmann-Schwinger equation): a periodic field on the
voxel grid is the Fourier series f(y) = sum_xi f_hat(xi) exp(i xi . y), so the
coefficients are

    f_hat[k] = (1/M) sum_n f[n] exp(-2 pi i k.n / N)        (``forward``)
    f[n]     =       sum_k f_hat[k] exp(+2 pi i k.n / N)     (``inverse``)

with M the number of voxels.  The voxel-centre offset of y only multiplies each
coefficient by a unit phase; every operator of the method is a Fourier
multiplier, so the offset cancels and index-based transforms are used.

Along an axis whose length is a power of two the transform is the textbook
recursive radix-2 decimation-in-time split; any other length (a factor of 3) uses
the DFT definition written out as a matrix product.  numpy.fft is never used here
(the tests use it only as an outside cross-check).

Pins: brute-force DFT with pure-Python loops on 4^3, 3^3, 6^3 and 2x3x4 grids,
Parseval, and numpy.fft (tests/test_oracle_fourier.py).
"""
import numpy as np

__all__ = ["dft_axis", "forward", "inverse", "frequencies", "discrete_frequencies",
           "wavevectors", "nyquist_mask"]


def _is_pow2(n):
    return n >= 1 and (n & (n - 1)) == 0


def _radix2_last(x, sign):
    """Recursive radix-2 DIT transform along the last axis (length a power of 2)."""
    n = x.shape[-1]
    if n == 1:
        return x.copy()
    even = _radix2_last(x[..., 0::2], sign)
    odd = _radix2_last(x[..., 1::2], sign)
    w = np.exp(sign * 2j * np.pi * np.arange(n // 2) / n)
    t = w * odd
    return np.concatenate([even + t, even - t], axis=-1)


def _naive_last(x, sign):
    """DFT definition along the last axis: X[k] = sum_n x[n] exp(sign 2 pi i n k / N)."""
    n = x.shape[-1]
    idx = np.arange(n)
    w = np.exp(sign * 2j * np.pi * np.outer(idx, idx) / n)
    return x @ w.T


def dft_axis(x, axis, sign):
    """Unnormalised DFT of ``x`` along ``axis`` with exponent sign ``sign`` (+1 or -1)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    y = _radix2_last(x, sign) if _is_pow2(x.shape[-1]) else _naive_last(x, sign)
    return np.moveaxis(y, -1, axis)


def forward(f):
    """Fourier coefficients over the last three axes (z, y, x), normalised by 1/M."""
    out = np.asarray(f, dtype=np.complex128)
    for ax in (-1, -2, -3):
        out = dft_axis(out, ax, -1)
    m = out.shape[-1] * out.shape[-2] * out.shape[-3]
    return out / m


def inverse(fh):
    """Sum of the Fourier series over the last three axes (unnormalised)."""
    out = np.asarray(fh, dtype=np.complex128)
    for ax in (-1, -2, -3):
        out = dft_axis(out, ax, +1)
    return out


def frequencies(n):
    """Integer frequency of each DFT index, in [-n/2, n/2) (Nyquist taken negative)."""
    j = np.arange(n)
    return np.where(j >= (n + 1) // 2, j - n, j)


def discrete_frequencies(n):
    """Integer frequency used for derivatives: ``frequencies`` with the Nyquist index set to 0.

    Reading of the paper on even grids: the sign of a Nyquist component is ambiguous
    (k = -N/2 and +N/2 alias), and neither Gamma0_hat nor the odd symbols are even in a
    single component, so a real operator needs a rule.  The derivative of a Nyquist
    mode is taken as zero (the average of its two signs), for every spectral operator.
    """
    k = frequencies(n)
    if n % 2 == 0:
        k = np.where(k == -(n // 2), 0, k)
    return k


def wavevectors(grid):
    """Discrete wave vector xi = 2 pi k / (N h) per axis, h = 1/max(N), Nyquist -> 0.

    ``grid`` is (N1, N2, N3) with N1 the fastest (x) axis.  Returns (xi1, xi2, xi3),
    each broadcastable to the array shape (N3, N2, N1).  Cubic voxels make the cubic
    grids exactly the unit torus of Sec. 2.
    """
    n1, n2, n3 = grid
    h = 1.0 / max(grid)
    xi1 = 2 * np.pi * discrete_frequencies(n1) / (n1 * h)
    xi2 = 2 * np.pi * discrete_frequencies(n2) / (n2 * h)
    xi3 = 2 * np.pi * discrete_frequencies(n3) / (n3 * h)
    return (xi1[None, None, :], xi2[None, :, None], xi3[:, None, None])


def nyquist_mask(grid):
    """True where any even axis sits at its Nyquist index N/2 (odd-symbol operators drop it)."""
    n1, n2, n3 = grid
    m = np.zeros((n3, n2, n1), dtype=bool)
    if n1 % 2 == 0:
        m[:, :, n1 // 2] = True
    if n2 % 2 == 0:
        m[:, n2 // 2, :] = True
    if n3 % 2 == 0:
        m[n3 // 2, :, :] = True
    return m
