"""Closed-form effective properties used to pin the oracle (test infrastructure).

None of these is the paper's method; they are textbook results the discrete
Lippmann-Schwinger solution must reproduce or respect:

* ``laminate_stiffness`` -- exact effective stiffness of a layered medium with normal
  e1.  With N = Mandel {11, 13, 12} (components carrying the traction on the layer
  planes) and T = {22, 33, 23} (in-plane strains, continuous across layers):
      C*_NN = <C_NN^-1>^-1,   C*_NT = C*_NN <C_NN^-1 C_NT>,
      C*_TT = <C_TT - C_TN C_NN^-1 C_NT> + <C_TN C_NN^-1> C*_NN <C_NN^-1 C_NT>.
  It is exact for voxel laminates solved with the Fourier scheme, because the only
  frequencies present are parallel to e1 and each layer's strain is constant.
* ``voigt`` / ``reuss`` -- arithmetic mean of C and harmonic mean of C.
* ``hs_bulk_bounds`` -- Hashin-Shtrikman bounds on the bulk modulus of a two-phase
  composite of isotropic phases.
* ``coated_cylinder_bulk`` / ``hashin_neutral_matrix_young`` -- Hashin's coated-cylinder
  assemblage (the structure of Sec. 4): its in-plane bulk modulus, and the matrix modulus that
  makes a coated inclusion neutral.  A neutral coated inclusion leaves a uniform hydrostatic
  field in the matrix undisturbed, so under in-plane hydrostatic strain the periodic cell of
  Sec. 4 has the matrix bulk modulus exactly (in the continuum).
"""
import numpy as np

from .tensors import iso_mandel_matrix

N_IDX = [0, 4, 5]
T_IDX = [1, 2, 3]


def laminate_stiffness(lame_layers, fractions):
    """Effective 6x6 Mandel stiffness of a laminate with normal e1.

    ``lame_layers`` is a list of (lambda, mu), ``fractions`` their volume fractions.
    """
    f = np.asarray(fractions, dtype=np.float64)
    f = f / f.sum()
    cs = [iso_mandel_matrix(l, m) for (l, m) in lame_layers]
    inv_nn = sum(fi * np.linalg.inv(c[np.ix_(N_IDX, N_IDX)]) for fi, c in zip(f, cs))
    cnn = np.linalg.inv(inv_nn)
    a = sum(fi * np.linalg.inv(c[np.ix_(N_IDX, N_IDX)]) @ c[np.ix_(N_IDX, T_IDX)]
            for fi, c in zip(f, cs))
    bt = sum(fi * c[np.ix_(T_IDX, N_IDX)] @ np.linalg.inv(c[np.ix_(N_IDX, N_IDX)])
             for fi, c in zip(f, cs))
    ctt0 = sum(fi * (c[np.ix_(T_IDX, T_IDX)]
                     - c[np.ix_(T_IDX, N_IDX)] @ np.linalg.inv(c[np.ix_(N_IDX, N_IDX)])
                     @ c[np.ix_(N_IDX, T_IDX)]) for fi, c in zip(f, cs))
    out = np.zeros((6, 6))
    out[np.ix_(N_IDX, N_IDX)] = cnn
    out[np.ix_(N_IDX, T_IDX)] = cnn @ a
    out[np.ix_(T_IDX, N_IDX)] = bt @ cnn
    out[np.ix_(T_IDX, T_IDX)] = ctt0 + bt @ cnn @ a
    return out


def voigt(lame_phases, fractions):
    f = np.asarray(fractions, dtype=np.float64)
    return sum(fi * iso_mandel_matrix(l, m) for fi, (l, m) in zip(f, lame_phases))


def reuss(lame_phases, fractions):
    f = np.asarray(fractions, dtype=np.float64)
    s = sum(fi * np.linalg.inv(iso_mandel_matrix(l, m)) for fi, (l, m) in zip(f, lame_phases))
    return np.linalg.inv(s)


def bulk(lam, mu):
    return lam + 2.0 * mu / 3.0


def hs_bulk_bounds(phase1, phase2, f2):
    """Hashin-Shtrikman (lower, upper) bulk modulus of two isotropic phases (lam, mu)."""
    k1, g1 = bulk(*phase1), phase1[1]
    k2, g2 = bulk(*phase2), phase2[1]
    f1 = 1.0 - f2
    if k1 > k2:
        (k1, g1, f1), (k2, g2, f2) = (k2, g2, f2), (k1, g1, f1)
    lower = k1 + f2 / (1.0 / (k2 - k1) + 3.0 * f1 / (3.0 * k1 + 4.0 * g1))
    upper = k2 + f1 / (1.0 / (k1 - k2) + 3.0 * f2 / (3.0 * k2 + 4.0 * g2))
    return lower, upper


def effective_bulk(c_eff):
    """Bulk modulus of a 6x6 Mandel stiffness under hydrostatic strain: (1/9) sum C_ij, i,j<3."""
    return float(np.sum(c_eff[:3, :3]) / 9.0)


def plane_stress_moduli(e, nu):
    """In-plane bulk and shear moduli of an isotropic plate in plane stress:
    kappa = E / (2 (1 - nu)) (mean in-plane stress over the trace of the in-plane strain) and
    mu = E / (2 (1 + nu))."""
    return e / (2.0 * (1.0 - nu)), e / (2.0 * (1.0 + nu))


def coated_cylinder_bulk(k_core, k_coat, mu_coat, f):
    """In-plane bulk modulus of Hashin's coated-cylinder assemblage with core fraction f (of the
    coated cylinder): kappa* = k2 + f / (1 / (k1 - k2) + (1 - f) / (k2 + mu2)), the classical
    composite-cylinder result in terms of two-dimensional bulk moduli."""
    return k_coat + f / (1.0 / (k_core - k_coat) + (1.0 - f) / (k_coat + mu_coat))


def hashin_neutral_matrix_young(e_core, e_coat, r1, r2, nu, plane_stress=True):
    """Young's modulus of the matrix that makes the coated disk (core r < r1, coating r < r2,
    common Poisson ratio nu) of Sec. 4 neutral: its two-dimensional bulk modulus equals the
    coated-cylinder bulk modulus with f = (r1 / r2)^2."""
    f = (r1 / r2) ** 2
    if plane_stress:
        k1, _ = plane_stress_moduli(e_core, nu)
        k2, mu2 = plane_stress_moduli(e_coat, nu)
        return 2.0 * (1.0 - nu) * coated_cylinder_bulk(k1, k2, mu2, f)
    # plane strain: kappa = lambda + mu = E / (2 (1 + nu) (1 - 2 nu))
    kp = lambda e: e / (2.0 * (1.0 + nu) * (1.0 - 2.0 * nu))
    mu2 = e_coat / (2.0 * (1.0 + nu))
    return 2.0 * (1.0 + nu) * (1.0 - 2.0 * nu) * coated_cylinder_bulk(kp(e_core), kp(e_coat), mu2, f)


def in_plane_bulk(c_eff):
    """In-plane bulk modulus (C11 + C22 + 2 C12) / 4 of a 6x6 Mandel stiffness (mean in-plane
    stress per unit in-plane trace under in-plane hydrostatic strain)."""
    return 0.25 * (c_eff[0, 0] + c_eff[1, 1] + c_eff[0, 1] + c_eff[1, 0])
