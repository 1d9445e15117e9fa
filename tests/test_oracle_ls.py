"""Pins of the oracle Lippmann-Schwinger operator and solvers (oracle/lippmann_schwinger.py)."""
import numpy as np
import pytest

from oracle import closed_forms, fourier
from oracle.lippmann_schwinger import Problem, assemble_A_mandel, gamma0_hat_slab, green_apply
from oracle.tensors import (iso_stiffness_4, iso_mandel_matrix, mandel_to_tensor,
                            tensor_to_mandel, unit_mandel_load, iso_apply, l2_norm)
from paper_1712_05145_gb300 import synthetic


def _random_xi(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3, n))


@pytest.mark.parametrize("lam0,mu0", [(5.5, 5.5), (0.0, 1.0), (2.3, 0.7), (-0.5, 2.0)])
def test_gamma_projection_identity(lam0, mu0):
    """Gamma0_hat : C0 : Gamma0_hat = Gamma0_hat at every xi != 0 (Sec. 2 Green operator)."""
    xi = _random_xi(20, 1)
    g = gamma0_hat_slab(xi[0], xi[1], xi[2], lam0, mu0)         # (3,3,3,3,20)
    c0 = iso_stiffness_4(lam0, mu0)
    gcg = np.einsum("ijmnz,mnpq,pqklz->ijklz", g, c0, g)
    np.testing.assert_allclose(gcg, g, atol=1e-14 * np.abs(g).max())


def test_gamma_symmetries_and_homogeneity():
    xi = _random_xi(10, 2)
    g = gamma0_hat_slab(xi[0], xi[1], xi[2], 2.0, 3.0)
    np.testing.assert_allclose(g, g.transpose(1, 0, 2, 3, 4), atol=1e-15)   # minor ij
    np.testing.assert_allclose(g, g.transpose(0, 1, 3, 2, 4), atol=1e-15)   # minor kl
    np.testing.assert_allclose(g, g.transpose(2, 3, 0, 1, 4), atol=1e-15)   # major
    g2 = gamma0_hat_slab(-3.7 * xi[0], -3.7 * xi[1], -3.7 * xi[2], 2.0, 3.0)
    np.testing.assert_allclose(g, g2, atol=1e-15)                           # even, degree 0
    z = gamma0_hat_slab(np.zeros(1), np.zeros(1), np.zeros(1), 2.0, 3.0)
    assert np.all(z == 0)


def test_gamma_annihilates_c0_constant_and_reproduces_compatible():
    """Gamma0 * (C0 : eps) = eps for a compatible zero-mean eps; Gamma0 * const = 0."""
    grid = (8, 6, 4)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((3, 4, 6, 8))
    from oracle.hierarchy import strain_from_displacement
    eps = strain_from_displacement(u, grid)
    lam0, mu0 = 1.3, 0.8
    c0e = iso_apply(lam0, mu0, eps)
    back = -fourier.inverse(green_apply(fourier.forward(c0e), grid, lam0, mu0)).real
    np.testing.assert_allclose(back, eps, atol=1e-12)
    const = np.ones((3, 3, 4, 6, 8))
    out = fourier.inverse(green_apply(fourier.forward(const), grid, lam0, mu0)).real
    assert np.abs(out).max() < 1e-14


def test_homogeneous_medium_gives_zero():
    ms = synthetic.centred_sphere(8, matrix=(2.0, 3.0), inclusion=(2.0, 3.0))
    pb = Problem(ms.phase, ms.lame, 2.0, 3.0)
    b = pb.rhs(unit_mandel_load(0))
    assert np.abs(b).max() < 1e-14
    pb2 = Problem(ms.phase, ms.lame, 7.0, 1.0)              # constant C != C0
    assert np.abs(pb2.rhs(unit_mandel_load(3))).max() < 1e-13


def test_polarization_forms_agree():
    """tau = (C-C0):eps + C:E and tau = (C-C0):(eps+E) give the same LS step (Gamma0 C0:E = 0)."""
    ms = synthetic.centred_sphere(8)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    rng = np.random.default_rng(7)
    eps = mandel_to_tensor(rng.standard_normal((6, 8, 8, 8)))
    E = mandel_to_tensor(rng.standard_normal(6))
    a = pb.ls_step(eps, E)
    ebig = np.broadcast_to(E[:, :, None, None, None], eps.shape)
    tau2 = iso_apply(pb.lam - pb.lam0, pb.mu - pb.mu0, eps + ebig)
    b = pb.minus_gamma_conv(tau2)
    np.testing.assert_allclose(a, b, atol=1e-13)


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 2)])
def test_solvers_match_dense_lu(shape):
    """Basic Scheme and CG reach the exact discrete solution (dense LU of A)."""
    rng = np.random.default_rng(11)
    phase = rng.integers(0, 3, size=shape).astype(np.uint8)
    lame = np.array([[1.0, 1.0], [4.0, 2.5], [0.5, 3.0]])
    pb = Problem(phase, lame, 2.0, 2.0)
    amat = assemble_A_mandel(pb)
    for a in (0, 4):
        b = pb.rhs(unit_mandel_load(a))
        x_lu = np.linalg.solve(amat, tensor_to_mandel(b).ravel()).reshape((6,) + shape)
        x_cg, _, _ = pb.cg(b, 1e-13)
        x_bs, _, _ = pb.basic_scheme(b, 1e-13)
        np.testing.assert_allclose(tensor_to_mandel(x_cg), x_lu, atol=1e-11)
        np.testing.assert_allclose(tensor_to_mandel(x_bs), x_lu, atol=1e-11)


def test_laminate_closed_form_worked_values():
    """Closed form at f = 1/2 with (1,1)/(10,10): exact fractions of the laminate formula."""
    c = closed_forms.laminate_stiffness([(1.0, 1.0), (10.0, 10.0)], [0.5, 0.5])
    # normal: harmonic mean of lam+2mu = (3, 30) -> 60/11; 1122 = 60/11 * <lam/(lam+2mu)> = 20/11
    assert abs(c[0, 0] - 60.0 / 11.0) < 1e-13
    assert abs(c[0, 1] - 20.0 / 11.0) < 1e-13 and abs(c[1, 0] - 20.0 / 11.0) < 1e-13
    # in-plane shear 23: arithmetic mean of 2 mu = 11; out-of-plane shears: harmonic = 40/11
    assert abs(c[3, 3] - 11.0) < 1e-13
    assert abs(c[4, 4] - 40.0 / 11.0) < 1e-13 and abs(c[5, 5] - 40.0 / 11.0) < 1e-13
    # 2222 = <lam+2mu - lam^2/(lam+2mu)> + <lam/(lam+2mu)>^2 * 60/11 = 168/11
    assert abs(c[1, 1] - 168.0 / 11.0) < 1e-12
    assert abs(c[1, 2] - 47.0 / 11.0) < 1e-12
    # single material: the formula returns that material
    one = closed_forms.laminate_stiffness([(2.0, 0.7), (2.0, 0.7)], [0.3, 0.7])
    np.testing.assert_allclose(one, iso_mandel_matrix(2.0, 0.7), atol=1e-13)


@pytest.mark.parametrize("scheme,split", [("cg", 2), ("basic", 4), ("cg", 6)])
def test_laminate_solution_is_exact(scheme, split):
    """Exact for layers of even thickness, whose strain has no Nyquist content along x1."""
    ms = synthetic.laminate((8, 4, 4), split=split)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    _, c_eff = pb.solve_order0(tol=1e-13, scheme=scheme)
    exact = closed_forms.laminate_stiffness([tuple(ms.lame[0]), tuple(ms.lame[1])],
                                            [split / 8, 1 - split / 8])
    np.testing.assert_allclose(c_eff, exact, atol=1e-10 * np.abs(exact).max())


def test_sphere_bounds_and_symmetry():
    ms = synthetic.centred_sphere(8)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    _, c_eff = pb.solve_order0(tol=1e-12)
    np.testing.assert_allclose(c_eff, c_eff.T, atol=1e-9 * np.abs(c_eff).max())   # major symmetry
    f = ms.volume_fractions()
    v = closed_forms.voigt([tuple(x) for x in ms.lame], f)
    r = closed_forms.reuss([tuple(x) for x in ms.lame], f)
    assert np.linalg.eigvalsh(v - c_eff).min() > -1e-10
    assert np.linalg.eigvalsh(c_eff - r).min() > -1e-10
    lo, hi = closed_forms.hs_bulk_bounds(tuple(ms.lame[0]), tuple(ms.lame[1]), f[1])
    k = closed_forms.effective_bulk(c_eff)
    assert lo <= k <= hi


@pytest.mark.parametrize("n", [8, 9])
def test_cg_result_independent_of_reference_medium(n):
    """Gamma0_hat(xi) is a C0-projection at every discrete xi, so the solution ignores C0."""
    ms = synthetic.centred_sphere(n)
    E = unit_mandel_load(1)
    outs = []
    for lam0, mu0 in [(5.5, 5.5), (0.0, 6.0), (3.0, 9.0)]:
        pb = Problem(ms.phase, ms.lame, lam0, mu0)
        eps, _, _ = pb.cg(pb.rhs(E), 1e-12)
        outs.append(eps)
    np.testing.assert_allclose(outs[1], outs[0], atol=1e-9)
    np.testing.assert_allclose(outs[2], outs[0], atol=1e-9)


def test_ls_step_is_a_real_operator():
    """The Fourier-series step maps real fields to real fields (Hermitian multiplier)."""
    ms = synthetic.centred_sphere(6)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    rng = np.random.default_rng(8)
    eps = mandel_to_tensor(rng.standard_normal((6, 6, 6, 6)))
    tau = pb.polarization(eps, None)
    full = fourier.inverse(green_apply(fourier.forward(tau), pb.grid, pb.lam0, pb.mu0))
    assert np.abs(full.imag).max() < 1e-13 * np.abs(full.real).max()
