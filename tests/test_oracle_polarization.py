"""Pins of the oracle's polarization scheme (oracle/polarization.py).

* Its fixed point is the exact discrete solution of A eps = b (Eq. cg_form): dense LU of the
  assembled operator on tiny grids, for the plain (relax = 1) and the averaged (relax = 1/2)
  iteration.
* Every plain step contracts the C0-energy-norm distance to the solution by at most
  q = max |(c - c0) / (c + c0)| over phases and Kelvin moduli, the rate the derivation gives.
* With the geometric-mean reference at contrast 100 it needs a fraction of the Basic Scheme's
  iterations; the averaged form converges at contrast 1e4.
"""
import numpy as np
import pytest

from oracle.lippmann_schwinger import Problem, assemble_A_mandel
from oracle import polarization as po
from oracle.tensors import c0_inner, tensor_to_mandel, unit_mandel_load
from paper_1712_05145_gb300 import synthetic

LAME = np.array([[1.0, 1.0], [4.0, 2.5], [0.5, 3.0]])


def problem(shape, lame, seed, reference):
    rng = np.random.default_rng(seed)
    phase = rng.integers(0, len(lame), size=shape).astype(np.uint8)
    lam0, mu0 = reference(lame)
    return Problem(phase, lame, lam0, mu0)


@pytest.mark.parametrize("relax", [1.0, 0.5])
@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 2)])
def test_fixed_point_is_the_dense_lu_solution(shape, relax):
    pb = problem(shape, LAME, 11, synthetic.geometric_reference)
    amat = assemble_A_mandel(pb)
    for a in (0, 4):
        b = pb.rhs(unit_mandel_load(a))
        x_lu = np.linalg.solve(amat, tensor_to_mandel(b).ravel()).reshape((6,) + shape)
        eps, it, _ = po.polarization_scheme(pb, LAME, b, relax=relax, tol=1e-14)
        np.testing.assert_allclose(tensor_to_mandel(eps), x_lu, atol=1e-11)
        assert it > 1


def test_each_step_contracts_by_the_predicted_factor():
    lame = np.array([[1.0, 1.0], [30.0, 20.0], [0.2, 0.1]])
    pb = problem((6, 4, 4), lame, 12, synthetic.midpoint_reference)   # a poor reference: q near 1
    q = po.contraction_factor(lame, pb.lam0, pb.mu0)
    assert 0.5 < q < 1.0
    b = pb.rhs(unit_mandel_load(1))
    xs = []
    po.polarization_scheme(pb, lame, b, relax=1.0, tol=1e-13, record=xs)
    xstar = xs[-1]
    err = [np.sqrt(c0_inner(x - xstar, x - xstar, pb.lam0, pb.mu0)) for x in xs[:-1]]
    ratios = [e1 / e0 for e0, e1 in zip(err[:20], err[1:21])]
    assert max(ratios) <= q * (1 + 1e-9), (max(ratios), q)
    assert max(ratios) > 0.5 * q        # the bound is approached, not trivially loose


def test_fewer_iterations_than_the_basic_scheme_at_contrast_100():
    lame = np.array([[1.0, 1.0], [100.0, 100.0]])
    pb_g = problem((8, 8, 8), lame, 13, synthetic.geometric_reference)
    pb_m = Problem(pb_g.phase, lame, *synthetic.midpoint_reference(lame))
    b_g = pb_g.rhs(unit_mandel_load(0))
    b_m = pb_m.rhs(unit_mandel_load(0))
    _, it_p, _ = po.polarization_scheme(pb_g, lame, b_g, tol=1e-8)
    _, it_b, _ = pb_m.basic_scheme(b_m, tol=1e-8)
    assert it_p < it_b / 3, (it_p, it_b)


def test_averaged_form_converges_at_contrast_1e4():
    lame = np.array([[1.0, 1.0], [1e4, 1e4]])
    pb = problem((4, 4, 4), lame, 14, synthetic.geometric_reference)
    amat = assemble_A_mandel(pb)
    b = pb.rhs(unit_mandel_load(5))
    x_lu = np.linalg.solve(amat, tensor_to_mandel(b).ravel()).reshape((6, 4, 4, 4))
    eps, _, _ = po.polarization_scheme(pb, lame, b, relax=0.5, tol=1e-13)
    np.testing.assert_allclose(tensor_to_mandel(eps), x_lu, atol=1e-9 * np.abs(x_lu).max())


def test_geometric_reference_minimises_the_contraction_factor():
    lame = np.array([[1.0, 1.0], [30.0, 20.0], [0.2, 0.1]])
    l0, m0 = synthetic.geometric_reference(lame)
    q = po.contraction_factor(lame, l0, m0)
    for dl, dm in ((0.05, 0), (-0.05, 0), (0, 0.05), (0, -0.05)):
        assert po.contraction_factor(lame, l0 * (1 + dl) + dl, m0 * (1 + dm)) >= q - 1e-12
