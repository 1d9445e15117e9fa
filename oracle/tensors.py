"""Oracle tensor algebra (test infrastructure; see ``oracle/__init__``).

Strain-like fields are full 3x3 tensors ``t[i, j, z, y, x]`` inside the oracle;
the Mandel vector (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12) is used only at the
boundary, so that a 6x6 Mandel matrix is the symmetric matrix of the quadratic
form and Frobenius products are plain dot products.

Hooke's law sigma = C : (eps + E) (Sec. 2, Eq. Hookes_law) with isotropic phases
C_ijkl = lambda d_ij d_kl + mu (d_ik d_jl + d_il d_jk) (same form as the reference
C0, Sec. 2), i.e. C : e = lambda tr(e) I + 2 mu e.

Pins: Mandel round trips and the 4-index stiffness against lambda tr(e) I + 2 mu e
(tests/test_oracle_tensors.py).
"""
import numpy as np

SQ2 = np.sqrt(2.0)
# Mandel index -> (i, j) and weight
MANDEL_PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
MANDEL_W = np.array([1.0, 1.0, 1.0, SQ2, SQ2, SQ2])


def mandel_to_tensor(v):
    """(6, ...) Mandel -> (3, 3, ...) symmetric tensor."""
    v = np.asarray(v)
    t = np.zeros((3, 3) + v.shape[1:], dtype=v.dtype)
    for a, (i, j) in enumerate(MANDEL_PAIRS):
        val = v[a] / MANDEL_W[a]
        t[i, j] = val
        t[j, i] = val
    return t


def tensor_to_mandel(t):
    """(3, 3, ...) tensor -> (6, ...) Mandel of its symmetric part."""
    t = np.asarray(t)
    out = np.empty((6,) + t.shape[2:], dtype=t.dtype)
    for a, (i, j) in enumerate(MANDEL_PAIRS):
        out[a] = MANDEL_W[a] * 0.5 * (t[i, j] + t[j, i])
    return out


def unit_mandel_load(a):
    """Macroscopic strain tensor E whose Mandel vector is the unit vector e_a."""
    v = np.zeros(6)
    v[a] = 1.0
    return mandel_to_tensor(v)


def iso_stiffness_4(lam, mu):
    """C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk) (Sec. 2, C0 formula)."""
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def iso_apply(lam, mu, e):
    """C : e for isotropic C with (possibly per-voxel) Lame fields lam, mu.

    ``e`` is (3, 3, ...) and lam, mu broadcast against the trailing axes.
    """
    tr = e[0, 0] + e[1, 1] + e[2, 2]
    out = 2.0 * mu * e
    for i in range(3):
        out[i, i] = out[i, i] + lam * tr
    return out


def iso_mandel_matrix(lam, mu):
    """6x6 Mandel matrix of an isotropic stiffness."""
    c = np.zeros((6, 6))
    c[:3, :3] = lam
    for i in range(3):
        c[i, i] += 2 * mu
    for i in range(3, 6):
        c[i, i] = 2 * mu
    return c


def ddot(a, b):
    """Pointwise a : b of two (3, 3, ...) fields."""
    return np.einsum("ij...,ij...->...", a, b)


def c0_inner(a, b, lam0, mu0):
    """<a, b>_C0 = mean( lam0 tr a tr b + 2 mu0 a : b ) = mean(a : C0 : b)."""
    tra = a[0, 0] + a[1, 1] + a[2, 2]
    trb = b[0, 0] + b[1, 1] + b[2, 2]
    return float(np.mean(lam0 * tra * trb + 2.0 * mu0 * ddot(a, b)))


def l2_norm(a):
    """Frobenius L2 norm with voxel mean: sqrt(mean(a : a))."""
    return float(np.sqrt(np.mean(ddot(a, a))))


def lame_fields(phase, lame_table):
    """Per-voxel (lambda, mu) from a phase array and an (n_phase, 2) Lame table."""
    tab = np.asarray(lame_table, dtype=np.float64)
    return tab[phase, 0], tab[phase, 1]
