"""Pins of the oracle's higher-order problems (oracle/hierarchy.py)."""
import numpy as np
import pytest

from oracle import fourier
from oracle.hierarchy import (Hierarchy, displacement_from_strain, strain_from_displacement,
                              theta_hat, rhs_order_alpha)
from oracle.lippmann_schwinger import Problem
from paper_1712_05145_gb300 import synthetic


@pytest.mark.parametrize("grid", [(8, 6, 4), (9, 3, 6)])
def test_theta_divergence_identity(grid):
    """i theta_hat(xi) xi = g_hat(xi) wherever the discrete wave vector is non-zero (Sec. 3)."""
    n1, n2, n3 = grid
    rng = np.random.default_rng(3)
    gh = fourier.forward(rng.standard_normal((3, n3, n2, n1)))
    th = theta_hat(gh, grid)
    xi1, xi2, xi3 = fourier.wavevectors(grid)
    xi = np.stack(np.broadcast_arrays(xi1, xi2, xi3))
    lhs = 1j * np.einsum("ij...,j...->i...", th, xi)
    keep = np.einsum("a...,a...->...", xi, xi) > 0
    assert keep.sum() > 0.5 * keep.size
    np.testing.assert_allclose(lhs[:, keep], gh[:, keep], atol=1e-14)
    np.testing.assert_allclose(th, np.swapaxes(th, 0, 1), atol=0)          # symmetric


@pytest.mark.parametrize("grid", [(8, 6, 4), (9, 12, 6)])
def test_displacement_strain_round_trip(grid):
    n1, n2, n3 = grid
    rng = np.random.default_rng(4)
    u0 = rng.standard_normal((3, n3, n2, n1))
    xi1, xi2, xi3 = fourier.wavevectors(grid)
    kill = (xi1 ** 2 + xi2 ** 2 + xi3 ** 2) == 0          # mean and pure-Nyquist modes
    assert kill.sum() == (1 + (n1 % 2 == 0)) * (1 + (n2 % 2 == 0)) * (1 + (n3 % 2 == 0))
    u_ref = fourier.inverse(np.where(kill, 0, fourier.forward(u0))).real
    eps = strain_from_displacement(u0, grid)
    np.testing.assert_allclose(displacement_from_strain(eps, grid), u_ref, atol=1e-12)
    # e_y of a linear-in-y displacement component: a single plane wave check
    y = np.arange(n1) / n1
    u1 = np.zeros((3, n3, n2, n1))
    u1[0] = np.sin(2 * np.pi * y)[None, None, :]
    e = strain_from_displacement(u1, grid)
    h = 1.0 / max(grid)
    np.testing.assert_allclose(e[0, 0], 2 * np.pi / (n1 * h) * np.cos(2 * np.pi * y)[None, None, :]
                               * np.ones((n3, n2, 1)), atol=1e-12)


def test_rhs_linear_in_p_and_g():
    ms = synthetic.centred_sphere(6)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    rng = np.random.default_rng(9)
    p1, p2 = rng.standard_normal((2, 3, 3, 6, 6, 6))
    p1 = 0.5 * (p1 + p1.swapaxes(0, 1))
    p2 = 0.5 * (p2 + p2.swapaxes(0, 1))
    g1, g2 = rng.standard_normal((2, 3, 6, 6, 6))
    a = rhs_order_alpha(pb, p1 + 2 * p2, g1 - g2)
    b = rhs_order_alpha(pb, p1, g1) + 2 * rhs_order_alpha(pb, p2, 0 * g2) - rhs_order_alpha(pb, 0 * p1, g2)
    np.testing.assert_allclose(a, b, atol=1e-13)


def test_order2_vanishes_for_centrosymmetric_cell():
    """alpha = 2 correctors are odd for a centrosymmetric cell, so D_1 = 0 to round-off."""
    ms = synthetic.centred_sphere(8)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    h = Hierarchy(pb, tol=1e-11)
    c = h.order1()
    d1 = h.order2()
    assert np.abs(d1).max() < 1e-8 * np.abs(c).max()
    # but the correctors themselves are not zero
    assert max(np.abs(e).max() for e in h.eps2.values()) > 1e-3


def test_order2_nonzero_for_asymmetric_cell_and_homogeneous_zero():
    rng = np.random.default_rng(12)
    phase = (rng.random((6, 6, 6)) < 0.4).astype(np.uint8)
    lame = np.array([[1.0, 1.0], [6.0, 4.0]])
    pb = Problem(phase, lame, 3.5, 2.5)
    h = Hierarchy(pb, tol=1e-11)
    h.order1()
    d1 = h.order2()
    assert np.abs(d1).max() > 1e-4
    hom = Problem(phase, np.array([[2.0, 1.0], [2.0, 1.0]]), 1.0, 1.5)
    hh = Hierarchy(hom, tol=1e-11)
    hh.order1()
    assert np.abs(hh.order2()).max() < 1e-12


# --- any order: the monomial-load builder ----------------------------------------------------

def _asym_small():
    from tests.helpers import random_phase
    g = (6, 4, 4)
    return synthetic.Microstructure(random_phase(g, 3, 21, p=[0.5, 0.3, 0.2]),
                                    np.array([[1.0, 1.0], [6.0, 4.0], [0.3, 0.2]]), 3.0, 2.0)


def test_monomial_derivatives():
    from oracle.hierarchy import derivative_value, monomial, multisets
    assert [len(multisets(d)) for d in range(5)] == [1, 3, 6, 10, 15]
    # d^K (Y^K / K!) = 1, and any other derivative of the same degree vanishes
    for K in multisets(3):
        for J in multisets(3):
            v = derivative_value(monomial(K), list(J))
            assert v == (1.0 if J == K else 0.0), (K, J, v)
    assert derivative_value(monomial((0, 0, 1)), [0]) is None   # still depends on Y


def test_general_builder_reproduces_orders_2_and_3():
    """The monomial-load builder gives the explicit alpha = 2 and alpha = 3 problems."""
    from oracle.hierarchy import GeneralHierarchy, multisets
    from oracle.tensors import MANDEL_PAIRS
    ms = _asym_small()
    h = Hierarchy(Problem(ms.phase, ms.lame, ms.lam0, ms.mu0), tol=1e-12)
    h.order1()
    h.order2()
    h.order3()
    G = GeneralHierarchy(h)
    np.testing.assert_allclose(G.solve(2), h.d1, rtol=0, atol=1e-13)
    idx = [6 * a + [i for i, pr in enumerate(MANDEL_PAIRS) if tuple(sorted(pr)) == K][0]
           for a in range(6) for K in multisets(2)]
    np.testing.assert_allclose(G.solve(3), h.d2[:, idx], rtol=0, atol=1e-13)


def test_order4_vanishes_for_centrosymmetric_cell_and_homogeneous_zero():
    """alpha = 4: the corrector is even for a centrosymmetric cell, so D_3 = 0 (as D_1); a
    homogeneous medium has zero correctors at every order."""
    from oracle.hierarchy import GeneralHierarchy
    ms = synthetic.centred_sphere(6)
    h = Hierarchy(Problem(ms.phase, ms.lame, ms.lam0, ms.mu0), tol=1e-12)
    h.order1()
    G = GeneralHierarchy(h)
    G.solve(2)
    d3 = G.solve(3)
    d4 = G.solve(4)
    assert np.abs(d3).max() > 1e-3
    assert np.abs(d4).max() < 1e-12 * np.abs(d3).max() * 1e3
    hom_ms = synthetic.Microstructure(np.zeros((4, 4, 4), np.uint8), np.array([[2.0, 1.0]]), 2.0, 1.0)
    h = Hierarchy(Problem(hom_ms.phase, hom_ms.lame, hom_ms.lam0, hom_ms.mu0), tol=1e-12)
    h.order1()
    G = GeneralHierarchy(h)
    for a in (2, 3, 4):
        assert np.abs(G.solve(a)).max() == 0.0
