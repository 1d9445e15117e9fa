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
