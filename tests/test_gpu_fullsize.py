"""Parity at the bench's full size (128^3, FP32 + refinement, the bench's launch configuration)
and properties that hold at any size on the 512^3 configuration.

* One LS step at 128^3 against the oracle, every element.
* The bench's solve: the oracle recomputes the FP64 residual and the equilibrium error of two
  GPU solutions with its own operator; C_eff is symmetric and lies between the Reuss and Voigt
  bounds.
* 512^3 Voronoi (256 grains): the reported FP64 residuals meet the tolerance, C_eff is symmetric
  and within the bounds of the voxel phase fractions.
"""
import os

import numpy as np
import pytest

from oracle import closed_forms
from oracle import equilibrium
from oracle.lippmann_schwinger import Problem
from oracle.tensors import mandel_to_tensor, tensor_to_mandel, unit_mandel_load
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL, oracle_ls_step_mandel, random_mandel_fields, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BENCH_GRID, BENCH_SEED, BENCH_TOL = 128, 1713, 1e-6


def bench_rve():
    return synthetic.random_spheres((BENCH_GRID,) * 3, seed=BENCH_SEED)


def between_bounds(c, lame, fractions, rel=1e-6):
    """C_eff - Reuss and Voigt - C_eff positive semi-definite (up to rel of the scale)."""
    v = closed_forms.voigt(lame, fractions)
    r = closed_forms.reuss(lame, fractions)
    cs = 0.5 * (c + c.T)
    scale = np.abs(v).max()
    return (np.linalg.eigvalsh(cs - r).min() > -rel * scale and np.linalg.eigvalsh(v - cs).min() > -rel * scale)


def test_ls_step_128_matches_oracle():
    from paper_1712_05145_gb300 import hom
    ms = bench_rve()
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    eps = random_mandel_fields(1, ms.grid, 17)
    E = np.random.default_rng(4).uniform(-1, 1, size=(1, 6))
    ref = oracle_ls_step_mandel(pb, eps[0], E[0])
    H = hom.Homogenization(ms, precision=hom.HOM_FP32_REFINE)
    ed = torch.from_numpy(eps).cuda()
    out = torch.empty_like(ed)
    hom.hom_ls_apply(H.h, 1, ed, E, out)
    assert rel_err(out.cpu().numpy()[0], ref) < TOL[1]
    H.close()


def test_bench_solve_residual_recomputed_by_oracle():
    from paper_1712_05145_gb300 import hom
    ms = bench_rve()
    H = hom.Homogenization(ms, precision=hom.HOM_FP32_REFINE, scheme=hom.HOM_CG)
    info = H.solve(0, BENCH_TOL)
    assert all(i["status"] == 0 and i["rel_residual_fp64"] < BENCH_TOL for i in info), info
    c = H.effective(0)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    eq_gpu = H.equilibrium_error()
    for a in (0, 3):
        E = unit_mandel_load(a)
        b = pb.rhs(E)
        eps = mandel_to_tensor(H.field(0, a))
        # the equilibrium error of the GPU solution, by the GPU and by the oracle
        eq_ref = equilibrium.equilibrium_error(equilibrium.stress_of(pb, eps, E), pb.grid)
        assert abs(eq_gpu[a] - eq_ref) < 1e-3 * eq_ref, (a, eq_gpu[a], eq_ref)
        res = pb.residual(eps, b)
        # the oracle's FP64 residual of the GPU solution meets the tolerance and agrees with the
        # residual the library reported (both FP64, different code)
        assert res < BENCH_TOL, (a, res)
        assert abs(res - info[a]["rel_residual_fp64"]) < 0.02 * res, (a, res, info[a])
        col = pb.mean_stress(eps, E)
        assert rel_err(c[:, a], col) < 1e-9
    assert np.abs(c - c.T).max() < 1e-5 * np.abs(c).max()
    assert between_bounds(c, [tuple(x) for x in ms.lame], ms.volume_fractions())
    H.close()


def test_voronoi_512_properties():
    from paper_1712_05145_gb300 import hom
    n = 512
    ms = synthetic.voronoi_torch((n, n, n), seed=1716, n_grains=256)   # phase on the device
    counts = torch.bincount(ms.phase.reshape(-1).long(), minlength=len(ms.lame)).cpu().numpy()
    fractions = counts / counts.sum()
    H = hom.Homogenization(ms, precision=hom.HOM_FP32_REFINE, scheme=hom.HOM_CG)
    info = H.solve(0, BENCH_TOL)
    assert all(i["status"] == 0 and i["rel_residual_fp64"] < BENCH_TOL for i in info), info
    c = H.effective(0)
    assert np.abs(c - c.T).max() < 1e-5 * np.abs(c).max()
    assert between_bounds(c, [tuple(x) for x in ms.lame], fractions)
    H.close()


def test_voronoi_128_solution_checked_by_oracle():
    """The Voronoi microstructure of the 512^3 configuration on a 128^3 grid (same seeds): the
    oracle recomputes the literal FP64 residual of the GPU solution for two loads."""
    from paper_1712_05145_gb300 import hom
    ms = synthetic.voronoi((128, 128, 128), seed=1716, n_grains=256)
    H = hom.Homogenization(ms, precision=hom.HOM_FP32_REFINE, scheme=hom.HOM_CG)
    info = H.solve(0, BENCH_TOL)
    assert all(i["status"] == 0 for i in info), info
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    for a in (1, 4):
        E = unit_mandel_load(a)
        res = pb.residual(mandel_to_tensor(H.field(0, a)), pb.rhs(E))
        assert res < BENCH_TOL, (a, res)
    c = H.effective(0)
    assert np.abs(c - c.T).max() < 1e-5 * np.abs(c).max()
    assert between_bounds(c, [tuple(x) for x in ms.lame], ms.volume_fractions())
    H.close()


GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STORED = {"random_spheres_128": lambda: synthetic.random_spheres((128, 128, 128), seed=1713),
          "voronoi_128": lambda: synthetic.voronoi((128, 128, 128), seed=1716, n_grains=256)}


@pytest.mark.parametrize("name", sorted(STORED))
def test_ceff_against_stored_oracle_solution(name):
    """C_eff of the two 128^3 configurations against the FP64 oracle's stored solution (its CG to a
    residual of 1e-10, written by tests/golden/make_ceff_golden.py): FP64 solves to 1e-11 agree
    within 1e-9, FP32 + refinement to 1e-9 within 1e-6, and at the throughput setting (residual
    1e-6) the error is bounded by 1e-4 (the bench states its value)."""
    import json
    from paper_1712_05145_gb300 import hom
    path = os.path.join(GOLDEN_DIR, "ceff_oracle_%s.json" % name)
    if not os.path.exists(path):
        pytest.skip("stored oracle solution not generated")
    with open(path) as f:
        ref = np.array(json.load(f)["c_eff"])
    ms = STORED[name]()
    for precision, tol, bound in ((hom.HOM_FP64, 1e-11, 1e-9), (hom.HOM_FP32_REFINE, 1e-9, 1e-6),
                                  (hom.HOM_FP32_REFINE, 1e-6, 1e-4)):
        H = hom.Homogenization(ms, precision=precision, scheme=hom.HOM_CG, max_iter=5000)
        info = H.solve(0, tol)
        assert all(i["status"] == 0 for i in info), (precision, tol, info)
        err = rel_err(H.effective(0), ref)
        H.close()
        assert err < bound, (precision, tol, err)
