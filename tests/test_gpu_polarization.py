"""GPU parity of the polarization scheme (Eyre-Milton / Monchiet-Bonnet and the averaged,
augmented-Lagrangian form) against oracle/polarization.py.

* Order 0 on a ragged 3-D grid and on a two-dimensional cell, both precisions, both variants:
  fields and C_eff against the oracle's fixed point; the literal FP64 residual certifies.
* Order 1 (right-hand sides from the order-0 correctors) against the oracle hierarchy.
* At contrast 100 it needs far fewer iterations than the Basic Scheme; a zero load is exact.
* Arguments that would make the scheme expand (non-positive reference moduli, an unknown
  variant) are rejected at creation.
"""
import numpy as np
import pytest

from oracle import polarization as po
from oracle.hierarchy import Hierarchy
from oracle.lippmann_schwinger import Problem
from oracle.tensors import tensor_to_mandel, unit_mandel_load
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL, TOL_EFF, random_phase, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAME = np.array([[1.0, 1.0], [6.0, 4.0], [0.3, 0.2]])


def cell(grid, seed):
    lam0, mu0 = synthetic.geometric_reference(LAME)
    return synthetic.Microstructure(random_phase(grid, 3, seed, p=[0.5, 0.3, 0.2]), LAME, lam0, mu0)


def oracle_polar(ms, loads, relax):
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    fields, cols = [], []
    for a in loads:
        E = unit_mandel_load(a)
        eps, _, _ = po.polarization_scheme(pb, ms.lame, pb.rhs(E), relax=relax, tol=1e-13)
        fields.append(tensor_to_mandel(eps))
        cols.append(pb.mean_stress(eps, E))
    return fields, np.stack(cols, axis=1)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("grid", [(16, 12, 6), (24, 8, 1)])
def test_order0_matches_oracle(grid, precision, variant):
    from paper_1712_05145_gb300 import hom
    ms = cell(grid, 51)
    ref_f, ref_c = oracle_polar(ms, range(6), 1.0 if variant == 0 else 0.5)
    H = hom.Homogenization(ms, precision=precision, scheme=hom.HOM_POLARIZATION, polarization_variant=variant)
    tol = 1e-12 if precision == 0 else 1e-9
    info = H.solve(0, tol)
    assert all(i["status"] == 0 and i["rel_residual_fp64"] < tol for i in info), info
    assert rel_err(H.effective(0), ref_c) < TOL_EFF[precision]
    for a in range(6):
        assert rel_err(H.field(0, a), ref_f[a]) < TOL[precision], a
    H.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_order1_matches_oracle_hierarchy(precision):
    from paper_1712_05145_gb300 import hom
    ms = cell((12, 8, 6), 53)
    h = Hierarchy(Problem(ms.phase, ms.lame, ms.lam0, ms.mu0), tol=1e-12)
    h.order1()
    h.order2()
    H = hom.Homogenization(ms, precision=precision, scheme=hom.HOM_POLARIZATION)
    tol = 1e-12 if precision == 0 else 1e-9
    for order in (0, 1):
        info = H.solve(order, tol)
        assert all(i["status"] == 0 for i in info), (order, info)
    assert rel_err(H.effective(0), h.c_eff) < TOL_EFF[precision]
    assert rel_err(H.effective(1), h.d1) < TOL_EFF[precision] * 10
    H.close()


def test_fewer_iterations_than_the_basic_scheme_at_contrast_100():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.random_spheres((32, 32, 32), seed=1713)
    geo = synthetic.geometric_reference(ms.lame)
    Hp = hom.Homogenization(ms, precision=0, scheme=hom.HOM_POLARIZATION, lam0=geo[0], mu0=geo[1])
    Hb = hom.Homogenization(ms, precision=0, scheme=hom.HOM_BASIC, max_iter=20000)
    ip = Hp.solve(0, 1e-6, loads=np.eye(6)[:1])[0]
    ib = Hb.solve(0, 1e-6, loads=np.eye(6)[:1])[0]
    assert ip["status"] == 0 and ib["status"] == 0
    assert ip["iterations"] < ib["iterations"] / 4, (ip, ib)
    assert rel_err(Hp.effective(0), Hb.effective(0)) < 1e-5
    Hp.close()
    Hb.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_load_is_exact(precision):
    from paper_1712_05145_gb300 import hom
    ms = cell((16, 12, 6), 55)
    H = hom.Homogenization(ms, precision=precision, scheme=hom.HOM_POLARIZATION)
    info = H.solve(0, 1e-10, loads=np.zeros((1, 6)))
    assert info[0]["status"] == 0 and info[0]["iterations"] == 0
    assert np.abs(H.field(0, 0)).max() == 0.0
    H.close()


def test_expanding_arguments_are_rejected():
    from paper_1712_05145_gb300 import hom
    ms = cell((16, 12, 6), 57)
    for lam0, mu0, variant in ((ms.lam0, -1.0, 0), (-1.0, 0.4, 0), (ms.lam0, ms.mu0, 2)):
        with pytest.raises(hom.HomError) as e:
            hom.Homogenization(ms, scheme=hom.HOM_POLARIZATION, lam0=lam0, mu0=mu0, polarization_variant=variant)
        assert e.value.status == hom.HOM_ERR_ARG


@pytest.mark.parametrize("precision", [0, 1])
def test_split_passes_match_fused(precision):
    """The polarization sweep through the split x and y passes gives the fused kernels' result."""
    from paper_1712_05145_gb300 import hom
    ms = cell((16, 12, 6), 59)
    tol = 1e-12 if precision == 0 else 1e-9
    out = []
    for pass_mode in (1, 2):
        H = hom.Homogenization(ms, precision=precision, scheme=hom.HOM_POLARIZATION, pass_mode=pass_mode)
        info = H.solve(0, tol)
        assert all(i["status"] == 0 for i in info), info
        out.append((H.effective(0), H.field(0, 2)))
        H.close()
    assert rel_err(out[1][0], out[0][0]) < TOL_EFF[precision]
    assert rel_err(out[1][1], out[0][1]) < TOL[precision]
