"""Pins of the oracle's equilibrium error (Sec. 2, Eq. eq_of_motion; oracle/equilibrium.py).

A stress that is constant plus cosine modes has an analytic divergence.  On a grid the modes
below the Nyquist frequency are resolved exactly, so the spectral definition must reproduce
both the closed form |A k| / (sqrt(2) |S|) and the voxel mean of the analytic |div sigma|^2
evaluated point by point (no transform).  k is the physical wave vector 2 pi m_i / L_i of the
cell with cubic voxels, L_i = N_i / max(N).
"""
import numpy as np
import pytest

from oracle import equilibrium as eq
from oracle.lippmann_schwinger import Problem
from oracle.tensors import mandel_to_tensor

GRID = (8, 6, 4)            # (N1, N2, N3): N1 fastest, arrays are (N3, N2, N1)


def sym(rng):
    a = rng.uniform(-1, 1, size=(3, 3))
    return a + a.T


def phase_of(m, grid):
    n1, n2, n3 = grid
    z, y, x = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    return 2 * np.pi * (m[0] * x / n1 + m[1] * y / n2 + m[2] * z / n3)


def wave(m, grid):
    """Physical wave vector of mode m: cubic voxels of size 1 / max(N)."""
    L = np.array(grid, dtype=float) / max(grid)
    return 2 * np.pi * np.asarray(m, dtype=float) / L


def field(S, terms, grid):
    """S + sum A cos(theta_m) (+ B sin) as a (3, 3, N3, N2, N1) array."""
    n1, n2, n3 = grid
    sig = np.broadcast_to(S[:, :, None, None, None], (3, 3, n3, n2, n1)).copy()
    for A, m, f in terms:
        sig += A[:, :, None, None, None] * f(phase_of(m, grid))[None, None]
    return sig


def brute_force(S, terms, grid):
    """sqrt(mean |div sigma|^2) / |<sigma>| with the analytic divergence at every voxel."""
    n1, n2, n3 = grid
    div = np.zeros((3, n3, n2, n1))
    for A, m, f in terms:
        k = wave(m, grid)
        df = (lambda t: -np.sin(t)) if f is np.cos else np.cos
        div += (A @ k)[:, None, None, None] * df(phase_of(m, grid))[None]
    return np.sqrt(np.mean(np.sum(div ** 2, axis=0))) / np.linalg.norm(S)


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 1, 1), (-1, 2, 1), (3, -2, 1)])
def test_single_mode_closed_form(m):
    rng = np.random.default_rng(sum(3 ** i * (v + 3) for i, v in enumerate(m)))
    S, A = sym(rng), sym(rng)
    got = eq.equilibrium_error(field(S, [(A, m, np.cos)], GRID), GRID)
    closed = np.linalg.norm(A @ wave(m, GRID)) / (np.sqrt(2.0) * np.linalg.norm(S))
    assert abs(got - closed) < 1e-12 * closed
    assert abs(got - brute_force(S, [(A, m, np.cos)], GRID)) < 1e-12 * closed


def test_two_modes_add_in_squares():
    rng = np.random.default_rng(5)
    S, A, B = sym(rng), sym(rng), sym(rng)
    m1, m2 = (1, 1, 0), (0, 2, 1)
    terms = [(A, m1, np.cos), (B, m2, np.sin)]
    got = eq.equilibrium_error(field(S, terms, GRID), GRID)
    closed = np.sqrt(0.5 * np.linalg.norm(A @ wave(m1, GRID)) ** 2
                     + 0.5 * np.linalg.norm(B @ wave(m2, GRID)) ** 2) / np.linalg.norm(S)
    assert abs(got - closed) < 1e-12 * closed
    assert abs(got - brute_force(S, terms, GRID)) < 1e-12 * closed


def test_homogeneous_and_zero_stress():
    rng = np.random.default_rng(6)
    S = sym(rng)
    assert eq.equilibrium_error(field(S, [], GRID), GRID) < 1e-13
    assert eq.equilibrium_error(np.zeros((3, 3, 4, 6, 8)), GRID) == 0.0


def test_nyquist_components_do_not_count():
    """Reading: the divergence uses the discrete wave vector, whose Nyquist components are 0."""
    rng = np.random.default_rng(7)
    S, A = sym(rng), sym(rng)
    # (-1)^n1: the pure x Nyquist mode is invisible
    assert eq.equilibrium_error(field(S, [(A, (4, 0, 0), np.cos)], GRID), GRID) < 1e-13
    # (-1)^n1 cos(2 pi n2 / 6): only the y component of the wave vector counts
    got = eq.equilibrium_error(field(S, [(A, (4, 1, 0), np.cos)], GRID), GRID)
    k = wave((0, 1, 0), GRID)
    closed = np.linalg.norm(A @ k) / (np.sqrt(2.0) * np.linalg.norm(S))
    assert abs(got - closed) < 1e-12 * closed


def test_zero_mean_stress_gives_the_unnormalised_norm():
    rng = np.random.default_rng(8)
    A = sym(rng)
    m = (1, 0, 1)
    got = eq.equilibrium_error(field(np.zeros((3, 3)), [(A, m, np.cos)], GRID), GRID)
    assert abs(got - np.linalg.norm(A @ wave(m, GRID)) / np.sqrt(2.0)) < 1e-12 * got


def test_solution_is_in_equilibrium_and_zero_strain_is_not():
    rng = np.random.default_rng(9)
    phase = rng.integers(0, 3, size=(4, 6, 8)).astype(np.uint8)
    lame = np.array([[1.0, 1.0], [8.0, 5.0], [0.3, 0.2]])
    pb = Problem(phase, lame, 3.0, 2.0)
    E = mandel_to_tensor(np.array([0.3, -0.2, 0.5, 0.1, 0.0, 0.4]))
    x, _, _ = pb.cg(pb.rhs(E), tol=1e-13)
    solved = eq.equilibrium_error(eq.stress_of(pb, x, E), GRID)
    unsolved = eq.equilibrium_error(eq.stress_of(pb, np.zeros_like(x), E), GRID)
    assert unsolved > 0.5
    assert solved < 1e-10 * unsolved
