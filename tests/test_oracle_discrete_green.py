"""Pins of the oracle's rotated finite-difference Green operator (oracle/discrete_green.py).

The operator is derived from a discretisation (averaged edge differences of corner
displacements), so its outside pin is that discretisation solved directly in real space: a
dense least-squares solve of D^T C (E + D u) = 0 assembled stencil by stencil.  A wrong sign,
index or factor in the symbol q, or in its use inside Gamma0_hat, changes the Lippmann-Schwinger
solution and fails it.  The symbol itself is checked against the stencil on plane waves, and the
scheme must reproduce the exact laminate stiffness for layer thicknesses where the spectral
operator with the Nyquist convention does not."""
import numpy as np
import pytest

from oracle import closed_forms, fourier
from oracle.discrete_green import (RotatedProblem, difference_matrix, real_space_solution, rotated_vectors)
from oracle.lippmann_schwinger import Problem, gamma0_hat_slab
from oracle.tensors import iso_stiffness_4, mandel_to_tensor, tensor_to_mandel, unit_mandel_load
from paper_1712_05145_gb300 import synthetic
from tests.helpers import random_phase, rel_err


def test_symbol_matches_the_difference_stencil_on_plane_waves():
    grid = (4, 6, 3)
    n1, n2, n3 = grid
    h = 1.0 / max(grid)
    D = difference_matrix(grid)
    m = n1 * n2 * n3
    q1, q2, q3 = np.broadcast_arrays(*rotated_vectors(grid))
    z, y, x = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    f1, f2, f3 = fourier.frequencies(n1), fourier.frequencies(n2), fourier.frequencies(n3)
    for (a, b, c) in [(1, 0, 0), (0, 2, 1), (2, 3, 1), (3, 5, 2)]:
        xi = np.array([2 * np.pi * f1[a] / (n1 * h), 2 * np.pi * f2[b] / (n2 * h), 2 * np.pi * f3[c] / (n3 * h)])
        corner = np.exp(1j * (xi[0] * x + xi[1] * y + xi[2] * z) * h).reshape(-1)
        centre = np.exp(1j * (xi[0] * (x + 0.5) + xi[1] * (y + 0.5) + xi[2] * (z + 0.5)) * h).reshape(-1)
        q = np.array([q1[c, b, a], q2[c, b, a], q3[c, b, a]])
        for d in range(3):
            u = np.zeros(3 * m, dtype=complex)
            u[d * m:(d + 1) * m] = corner
            eps = D @ u
            # the normal strain of displacement component d is D_d u_d
            got = eps[d * m:(d + 1) * m]
            assert np.allclose(got, (2j / h) * q[d] * centre, atol=1e-10)


@pytest.mark.parametrize("grid,nphase,seed", [((4, 4, 4), 3, 1), ((3, 4, 2), 2, 2), ((4, 6, 2), 3, 3)])
def test_lippmann_schwinger_solution_equals_real_space_solve(grid, nphase, seed):
    lame = np.array([[1.0, 0.8], [9.0, 6.0], [0.3, 0.5]])[:nphase]
    phase = random_phase(grid, nphase, seed)
    pb = RotatedProblem(phase, lame, 4.0, 3.0)
    for a in (0, 3, 5):
        E = unit_mandel_load(a)
        eps, _, _ = pb.cg(pb.rhs(E), 1e-13)
        ref = real_space_solution(phase, lame, np.eye(6)[a])
        assert rel_err(tensor_to_mandel(eps), ref) < 1e-9, a
    # the spectral operator solves a different discrete problem
    sp = Problem(phase, lame, 4.0, 3.0)
    eps_sp, _, _ = sp.cg(sp.rhs(unit_mandel_load(0)), 1e-13)
    assert rel_err(tensor_to_mandel(eps_sp), real_space_solution(phase, lame, np.eye(6)[0])) > 1e-4


def test_rotated_green_is_a_C0_projection_and_vanishes_where_q_does():
    grid = (4, 6, 8)
    lam0, mu0 = 2.0, 1.5
    q1, q2, q3 = np.broadcast_arrays(*rotated_vectors(grid))
    C0 = iso_stiffness_4(lam0, mu0)
    zero = 0
    for idx in np.ndindex(q1.shape):
        g = gamma0_hat_slab(q1[idx], q2[idx], q3[idx], lam0, mu0)
        qq = q1[idx] ** 2 + q2[idx] ** 2 + q3[idx] ** 2
        if qq == 0.0:
            zero += 1
            assert np.abs(g).max() == 0.0
            continue
        gcg = np.einsum("ijkl,klmn,mnpq->ijpq", g, C0, g)
        assert np.abs(gcg - g).max() < 1e-12
    assert zero == _count_q_zero(grid) == 17   # the mean and the 16 frequencies with two or more Nyquist indices


def _count_q_zero(grid):
    q1, q2, q3 = np.broadcast_arrays(*rotated_vectors(grid))
    return int(np.sum(q1 ** 2 + q2 ** 2 + q3 ** 2 == 0.0))


def test_strain_free_frequencies():
    """q = 0 exactly at the mean and where at least two axes sit at their Nyquist index."""
    for grid in [(4, 6, 8), (4, 4, 3), (3, 5, 7)]:
        n1, n2, n3 = grid
        ny = [n % 2 == 0 for n in grid]
        expected = 1
        # pairs of Nyquist axes with the third axis free, minus double counting of all three
        free = [n1, n2, n3]
        pairs = [(0, 1, 2), (0, 2, 1), (1, 2, 0)]
        for i, j, k in pairs:
            if ny[i] and ny[j]:
                expected += free[k]
        if all(ny):
            expected -= 2   # the all-Nyquist frequency is counted in three pairs
        assert _count_q_zero(grid) == expected, grid


def test_laminate_is_exact_for_any_layer_thickness():
    """Fields of a laminate normal to y1 depend on y1 only; the difference scheme represents the
    piecewise-constant strain exactly, so C_eff is the closed form for 5 + 11 layers, which the
    spectral operator (Nyquist convention) misses."""
    ms = synthetic.laminate((16, 4, 4), split=5, a=(1.0, 1.0), b=(10.0, 10.0))
    fr = ms.volume_fractions()
    exact = closed_forms.laminate_stiffness([tuple(x) for x in ms.lame], fr)
    pb = RotatedProblem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    _, c = pb.solve_order0(tol=1e-13)
    assert rel_err(c, exact) < 1e-10
    sp = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    _, c_sp = sp.solve_order0(tol=1e-13)
    assert rel_err(c_sp, exact) > 1e-6


def test_solution_does_not_depend_on_the_reference_medium():
    grid = (6, 4, 4)
    lame = np.array([[1.0, 1.0], [20.0, 12.0]])
    phase = random_phase(grid, 2, 5)
    sols = []
    for lam0, mu0 in ((10.0, 6.0), (3.0, 9.0)):
        pb = RotatedProblem(phase, lame, lam0, mu0)
        eps, _, _ = pb.cg(pb.rhs(unit_mandel_load(1)), 1e-13)
        sols.append(eps)
    assert rel_err(sols[0], sols[1]) < 1e-10
