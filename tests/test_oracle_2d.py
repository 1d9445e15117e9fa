"""Two-dimensional cells (N3 = 1) and Hashin's structure of Sec. 4: pins of the oracle.

* The matrix modulus the paper prints for its Hashin structure (tests/golden) follows from the
  coated-cylinder closed form in plane stress, which fixes the two-dimensional reading.
* A cell with N3 = 1 is the z-extrusion of itself: the oracle gives the same fields and C_eff
  on (N1, N2, 1) as on the (N1, N2, 2) grid with both planes equal.
* A plane-stress voxel laminate has the exact laminate stiffness (in-plane block).
* The neutral coated inclusion gives the matrix bulk modulus under grid refinement.
"""
import os

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import lippmann_schwinger as ls
from oracle.tensors import mandel_to_tensor
from paper_1712_05145_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hashin_2d_neutral_matrix.txt")
IN_PLANE = [0, 1, 5]   # Mandel 11, 22, 12


def golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_neutral_matrix_modulus_is_the_papers():
    g = golden()
    e3 = cf.hashin_neutral_matrix_young(g["E1"], g["E2"], g["r1"], g["r2"], g["nu"], plane_stress=True)
    assert abs(e3 - g["E3"]) < 5e-4          # printed to three decimals
    # the plane-strain reading does not give the printed value
    e3_strain = cf.hashin_neutral_matrix_young(g["E1"], g["E2"], g["r1"], g["r2"], g["nu"], plane_stress=False)
    assert abs(e3_strain - g["E3"]) > 10.0


def test_plane_stress_lame_reproduces_plane_stress_law():
    lam, mu = synthetic.lame_from_young(7.0, 0.3)
    ls_, mu_ = synthetic.plane_stress_lame(lam, mu)
    k, m = cf.plane_stress_moduli(7.0, 0.3)
    assert abs((ls_ + mu_) - k) < 1e-12 and abs(mu_ - m) < 1e-12
    # sigma33 = 0 in plane stress: eps33 = -lam/(lam+2mu) tr2, and sigma11 = lam* tr2 + 2 mu eps11
    e11, e22 = 0.3, -0.7
    e33 = -lam / (lam + 2 * mu) * (e11 + e22)
    s11 = lam * (e11 + e22 + e33) + 2 * mu * e11
    assert abs(s11 - (ls_ * (e11 + e22) + 2 * mu_ * e11)) < 1e-12


def _c_eff(phase, lame, lam0, mu0):
    P = ls.Problem(phase, lame, lam0, mu0)
    sols, c = P.solve_order0(tol=1e-12)
    return sols, c


def test_two_dimensional_cell_equals_its_extrusion():
    rng = np.random.default_rng(12)
    phase = rng.integers(0, 3, size=(1, 6, 8)).astype(np.uint8)
    lame = np.array([[1.0, 1.0], [6.0, 3.0], [0.4, 0.3]])
    lam0, mu0 = synthetic.midpoint_reference(lame)
    s1, c1 = _c_eff(phase, lame, lam0, mu0)
    s2, c2 = _c_eff(np.repeat(phase, 2, axis=0), lame, lam0, mu0)
    np.testing.assert_allclose(c1, c2, rtol=0, atol=1e-10 * np.abs(c2).max())
    for a, b in zip(s1, s2):
        np.testing.assert_allclose(a[..., 0, :, :], b[..., 1, :, :], rtol=0, atol=1e-10)


def test_plane_stress_laminate_closed_form():
    layers = [synthetic.plane_stress_lame(*synthetic.lame_from_young(e, nu)) for e, nu in ((1.0, 0.3), (20.0, 0.25))]
    ms = synthetic.laminate((8, 8, 1), a=layers[0], b=layers[1])
    _, c = _c_eff(ms.phase, ms.lame, ms.lam0, ms.mu0)
    ref = cf.laminate_stiffness(layers, [0.5, 0.5])
    blk = np.ix_(IN_PLANE, IN_PLANE)
    np.testing.assert_allclose(c[blk], ref[blk], rtol=0, atol=1e-10 * np.abs(ref).max())


def test_hashin_bulk_converges_to_matrix_bulk():
    g = golden()
    k3, _ = cf.plane_stress_moduli(g["E3"], g["nu"])
    E = mandel_to_tensor(np.array([1.0, 1.0, 0, 0, 0, 0]))
    err = []
    for n in (16, 32, 64):
        ms = synthetic.hashin_2d(n)
        P = ls.Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
        _, c = P.solve_order0(tol=1e-10, loads=[E])
        err.append(abs(0.25 * (c[0, 0] + c[1, 0]) - k3) / k3)
    assert err[2] < err[1] < err[0]
    assert err[2] < 0.015
