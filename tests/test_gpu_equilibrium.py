"""GPU parity of the equilibrium error (Sec. 2, Eq. eq_of_motion) against the oracle.

* Arbitrary strain fields and loads: every value against oracle/equilibrium.py, on a 3-D grid
  whose half spectrum spans several CTAs with a ragged tail, on a two-dimensional cell, and
  with the split x and y passes, in both precisions.
* Solved order-0 loads: the GPU's value for its own solution matches the oracle's value for
  the same field, and is far below the value of the unsolved field (eps = 0).
* Degenerate and error cases: zero stress, order 0 not solved, a wrong load count.
"""
import numpy as np
import pytest

from oracle import equilibrium as eq
from oracle.lippmann_schwinger import Problem
from oracle.tensors import mandel_to_tensor
from paper_1712_05145_gb300 import synthetic
from tests.helpers import random_mandel_fields, random_phase

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# double transforms: rounding of a few ulps; double-float transforms (FP32 mode): about 2^-44
TOL_RANDOM = {0: 1e-11, 1: 1e-9}
LAME = np.array([[1.0, 1.0], [6.0, 4.0], [0.3, 0.2]])


def cell(grid, seed):
    return synthetic.Microstructure(random_phase(grid, 3, seed, p=[0.5, 0.3, 0.2]), LAME, 3.0, 2.0)


def oracle_values(ms, eps, E):
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    grid = (ms.phase.shape[2], ms.phase.shape[1], ms.phase.shape[0])
    return np.array([eq.equilibrium_error(eq.stress_of(pb, mandel_to_tensor(eps[l]), mandel_to_tensor(E[l])), grid)
                     for l in range(eps.shape[0])])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("grid,pass_mode", [((16, 12, 6), 0), ((24, 8, 1), 0), ((16, 12, 6), 2)])
def test_random_fields_match_oracle(precision, grid, pass_mode):
    from paper_1712_05145_gb300 import hom
    ms = cell(grid, 41)
    eps = random_mandel_fields(3, grid, 43)
    E = np.random.default_rng(44).uniform(-1, 1, size=(3, 6))
    ref = oracle_values(ms, eps, E)
    H = hom.Homogenization(ms, precision=precision, pass_mode=pass_mode)
    got = hom.hom_equilibrium_error(H.h, 3, torch.from_numpy(eps).cuda(), E)
    assert np.all(ref > 1.0)
    assert np.max(np.abs(got - ref) / ref) < TOL_RANDOM[precision], (got, ref)
    H.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_solved_loads_match_oracle(precision):
    from paper_1712_05145_gb300 import hom
    grid = (16, 12, 6)
    ms = cell(grid, 45)
    tol = 1e-10 if precision == 0 else 1e-8
    H = hom.Homogenization(ms, precision=precision)
    info = H.solve(0, tol)
    assert all(i["status"] == 0 for i in info)
    got = H.equilibrium_error()
    assert got.shape == (6,)
    eps = np.stack([H.field(0, a) for a in range(6)])
    ref = oracle_values(ms, eps, np.eye(6))
    assert np.max(np.abs(got - ref) / ref) < 1e-3, (got, ref)
    # the unsolved field eps = 0 is far from equilibrium
    unsolved = hom.hom_equilibrium_error(H.h, 6, torch.zeros((6, 6, 6, 12, 16), dtype=torch.float64,
                                                               device="cuda"), np.eye(6))
    assert np.all(got < 1e-4 * unsolved), (got, unsolved)
    H.close()


def test_zero_stress_and_errors():
    from paper_1712_05145_gb300 import hom
    grid = (16, 12, 6)
    ms = cell(grid, 47)
    H = hom.Homogenization(ms, precision=0)
    z = torch.zeros((2, 6, 6, 12, 16), dtype=torch.float64, device="cuda")
    assert np.all(hom.hom_equilibrium_error(H.h, 2, z, None) == 0.0)
    with pytest.raises(hom.HomError) as e:
        hom.hom_equilibrium_error(H.h, 6)
    assert e.value.status == hom.HOM_ERR_ORDER
    H.solve(0, 1e-10, loads=np.eye(6)[:2])
    with pytest.raises(hom.HomError) as e:
        hom.hom_equilibrium_error(H.h, 3)
    assert e.value.status == hom.HOM_ERR_ARG
    assert H.equilibrium_error().shape == (2,)
    H.close()


def test_unit_load_on_a_homogeneous_cell_is_in_equilibrium():
    """One phase: sigma = C : E is constant, so the error is 0 up to rounding."""
    from paper_1712_05145_gb300 import hom
    ms = synthetic.Microstructure(np.zeros((6, 12, 16), dtype=np.uint8), LAME[:1], 1.5, 1.2)
    H = hom.Homogenization(ms, precision=0)
    z = torch.zeros((1, 6, 6, 12, 16), dtype=torch.float64, device="cuda")
    got = hom.hom_equilibrium_error(H.h, 1, z, np.eye(6)[3:4])
    assert got[0] < 1e-13
    H.close()
