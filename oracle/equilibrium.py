"""Oracle equilibrium error of a stress field (test infrastructure; see ``oracle/__init__``).

Sec. 2 of arXiv:1712.05145: the stress sigma = C : (eps + E) (Eq. Hookes_law) of a solution
satisfies the balance of momentum div sigma = 0 (Eq. eq_of_motion).  The paper notes that
convergence criteria other than its Cauchy quantity are possible; this module measures the
distance from equilibrium in the form Moulinec and Suquet use (the paper's reference for the
Basic Scheme):

    e = sqrt(< |div sigma|^2 >) / |<sigma>|

with <.> the voxel mean, |.| the Frobenius norm, and the divergence taken term by term on the
Fourier series of ``fourier`` (coefficients normalised by 1/M):
(div sigma)_hat(xi) = i xi . sigma_hat(xi) with the discrete wave vectors of the Green operator
(``fourier.wavevectors``, Nyquist components 0).  By Parseval
<|div sigma|^2> = sum over all xi of |xi . sigma_hat(xi)|^2 and <sigma> = sigma_hat(0).
Reading for the degenerate case: where the mean stress vanishes up to rounding,
|<sigma>| <= 1e-12 sqrt(<|sigma|^2>) (a zero load), the error is sqrt(<|div sigma|^2>) itself,
and 0 for sigma = 0.

Pins (tests/test_oracle_equilibrium.py): a constant stress plus one cosine mode has the closed
form |A k| / (sqrt(2) |S|) with k the mode's physical wave vector, along each axis of a
non-cubic grid and for an off-axis mode; two modes at different frequencies add in squares; a
homogeneous stress gives 0, and so does a mode at the Nyquist frequency (its discrete wave
vector component is 0); the oracle's own converged solution of a heterogeneous cell gives an
error at the level of its tolerance, while eps = 0 on the same cell does not.
"""
import numpy as np

from . import fourier

__all__ = ["divergence_hat", "equilibrium_error", "stress_of", "ZERO_MEAN"]

ZERO_MEAN = 1e-12      # |<sigma>| / sqrt(<|sigma|^2>) at or below which the mean counts as 0


def stress_of(problem, eps, E):
    """sigma = C : (eps + E) for a (3, 3, N3, N2, N1) strain fluctuation and a 3x3 load E."""
    ebig = np.broadcast_to(E.reshape(E.shape + (1,) * (eps.ndim - 2)), eps.shape)
    return problem.stress(eps + ebig)


def divergence_hat(sigma_hat, grid):
    """Fourier coefficients of div sigma: i xi_j sigma_hat_ij over the discrete xi."""
    xi = fourier.wavevectors(grid)
    return np.stack([1j * sum(sigma_hat[i, j] * xi[j] for j in range(3)) for i in range(3)])


def equilibrium_error(sigma, grid):
    """e = sqrt(<|div sigma|^2>) / |<sigma>| for a (3, 3, N3, N2, N1) stress field."""
    sigma_hat = fourier.forward(sigma)
    d = divergence_hat(sigma_hat, grid)
    num = np.sqrt(np.sum(np.abs(d) ** 2))
    den = np.sqrt(np.sum(np.abs(sigma_hat[:, :, 0, 0, 0]) ** 2))
    rms = np.sqrt(np.mean(np.sum(sigma ** 2, axis=(0, 1))))
    return float(num / den) if den > ZERO_MEAN * rms else float(num)
