"""GPU parity of the higher-order problems (orders 1 to 6, the paper's alpha = 2 to 7)."""
import numpy as np
import pytest

from oracle.hierarchy import Hierarchy
from oracle.lippmann_schwinger import Problem
from oracle.tensors import tensor_to_mandel
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL, TOL_EFF, random_phase, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def asym_cell():
    g = (8, 12, 6)
    return synthetic.Microstructure(random_phase(g, 3, 21, p=[0.5, 0.3, 0.2]),
                                    np.array([[1.0, 1.0], [6.0, 4.0], [0.3, 0.2]]), 3.0, 2.0)


@pytest.fixture(scope="module")
def oracle_asym():
    ms = asym_cell()
    h = Hierarchy(Problem(ms.phase, ms.lame, ms.lam0, ms.mu0), tol=1e-12)
    h.order1()
    h.order2()
    h.order3()
    return ms, h


@pytest.mark.parametrize("precision", [0, 1])
def test_orders_0_1_2_match_oracle(oracle_asym, precision):
    from paper_1712_05145_gb300 import hom
    ms, oh = oracle_asym
    H = hom.Homogenization(ms, precision=precision)
    tol = 1e-12 if precision == 0 else 1e-9
    for order in (0, 1, 2):
        info = H.solve(order, tol)
        assert all(i["status"] == 0 for i in info), (order, info)
    tol_f = TOL[precision] * (1 if precision == 0 else 5)
    assert rel_err(H.effective(0), oh.c_eff) < TOL_EFF[precision]
    assert rel_err(H.effective(1), oh.d1) < TOL_EFF[precision] * 10
    assert rel_err(H.effective(2), oh.d2) < TOL_EFF[precision] * 10
    for a in (0, 4):
        assert rel_err(H.field(0, a, hom.HOM_FIELD_DISPLACEMENT), oh.chi[a]) < tol_f
    for L in (0, 7, 17):
        a, k = divmod(L, 3)
        assert rel_err(H.field(1, L), tensor_to_mandel(oh.eps2[(a, k)])) < tol_f, L
        assert rel_err(H.field(1, L, hom.HOM_FIELD_DISPLACEMENT), oh.u2[(a, k)]) < tol_f, L
    for L in (0, 11, 35):
        a, P = divmod(L, 6)
        assert rel_err(H.field(2, L), tensor_to_mandel(oh.eps3[(a, P)])) < tol_f, L
    H.close()


def test_order1_vanishes_for_centrosymmetric_cell():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.centred_sphere(16)
    H = hom.Homogenization(ms, precision=0)
    H.solve(0, 1e-12)
    info = H.solve(1, 1e-12)
    assert all(i["status"] == 0 for i in info)
    d1 = H.effective(1)
    assert np.abs(d1).max() < 1e-9 * np.abs(H.effective(0)).max()
    assert np.abs(H.field(1, 4)).max() > 1e-4
    H.close()


def test_order_dependencies_enforced():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.centred_sphere(8)
    H = hom.Homogenization(ms, precision=0)
    with pytest.raises(hom.HomError) as e:
        H.solve(1, 1e-8)
    assert e.value.status == hom.HOM_ERR_ORDER
    H.solve(0, 1e-10, loads=np.eye(6)[:2])
    with pytest.raises(hom.HomError):
        H.solve(1, 1e-8)
    H.close()


@pytest.fixture(scope="module")
def oracle_general(oracle_asym):
    from oracle.hierarchy import GeneralHierarchy
    ms, oh = oracle_asym
    G = GeneralHierarchy(oh)
    for alpha in (2, 3, 4, 5):
        G.solve(alpha)
    return ms, G


@pytest.mark.parametrize("precision", [0, 1])
def test_orders_3_and_4_match_oracle(oracle_general, precision):
    """Orders 3 and 4 (the paper's alpha = 4, 5) from the recursive right-hand-side builder."""
    from oracle.hierarchy import multisets
    from paper_1712_05145_gb300 import hom
    ms, G = oracle_general
    H = hom.Homogenization(ms, precision=precision)
    tol = 1e-12 if precision == 0 else 1e-9
    for order in range(5):
        info = H.solve(order, tol)
        assert len(info) == hom.loads_of_order(order)
        assert all(i["status"] == 0 for i in info), (order, info)
    tol_f = TOL[precision] * (1 if precision == 0 else 10)
    for order in (3, 4):
        D = H.effective(order)
        assert rel_err(D, G.D[order + 1]) < TOL_EFF[precision] * 10, order
        Ks = multisets(order)
        for L in (0, len(Ks) + 3, 6 * len(Ks) - 1):
            a, k = divmod(L, len(Ks))
            ref = tensor_to_mandel(G.eps[order + 1][(a, Ks[k])])
            assert rel_err(H.field(order, L), ref) < tol_f, (order, L)
    H.close()


def test_order3_vanishes_for_centrosymmetric_cell():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.centred_sphere(16)
    H = hom.Homogenization(ms, precision=0)
    for order in range(4):
        info = H.solve(order, 1e-12)
        assert all(i["status"] == 0 for i in info)
    assert np.abs(H.effective(3)).max() < 1e-9 * np.abs(H.effective(2)).max()
    assert np.abs(H.effective(2)).max() > 1e-4
    H.close()


@pytest.fixture(scope="module")
def oracle_general_small():
    """An asymmetric three-phase 4 x 6 x 4 cell with the oracle's orders up to alpha = 7."""
    from oracle.hierarchy import GeneralHierarchy
    g = (4, 6, 4)
    ms = synthetic.Microstructure(random_phase(g, 3, 23, p=[0.5, 0.3, 0.2]),
                                  np.array([[1.0, 1.0], [6.0, 4.0], [0.3, 0.2]]), 3.0, 2.0)
    h = Hierarchy(Problem(ms.phase, ms.lame, ms.lam0, ms.mu0), tol=1e-12)
    h.order1()
    h.order2()
    G = GeneralHierarchy(h)
    for alpha in range(2, 8):
        G.solve(alpha)
    return ms, G


@pytest.mark.parametrize("precision", [0, 1])
def test_orders_5_and_6_match_oracle(oracle_general_small, precision):
    """Orders 5 and 6 (the paper's alpha = 6, 7): 126 and 168 unit loads."""
    from oracle.hierarchy import multisets
    from paper_1712_05145_gb300 import hom
    ms, G = oracle_general_small
    H = hom.Homogenization(ms, precision=precision)
    tol = 1e-12 if precision == 0 else 1e-9
    for order in range(7):
        info = H.solve(order, tol)
        assert len(info) == hom.loads_of_order(order)
        assert all(i["status"] == 0 for i in info), (order, info)
    tol_f = TOL[precision] * (1 if precision == 0 else 10)
    for order in (5, 6):
        D = H.effective(order)
        assert D.shape == (6, hom.loads_of_order(order))
        assert rel_err(D, G.D[order + 1]) < TOL_EFF[precision] * 10, order
        Ks = multisets(order)
        for L in (0, len(Ks) + 5, 6 * len(Ks) - 1):
            a, k = divmod(L, len(Ks))
            ref = tensor_to_mandel(G.eps[order + 1][(a, Ks[k])])
            assert rel_err(H.field(order, L), ref) < tol_f, (order, L)
    with pytest.raises(hom.HomError) as e:
        H.solve(7, tol)
    assert e.value.status == hom.HOM_ERR_ARG
    H.close()


def test_order5_vanishes_for_centrosymmetric_cell():
    """D5 (alpha = 6) is an odd-order tensor: zero for a centrosymmetric cell, like D1 and D3."""
    from paper_1712_05145_gb300 import hom
    ms = synthetic.centred_sphere(8)
    H = hom.Homogenization(ms, precision=0)
    for order in range(6):
        info = H.solve(order, 1e-12)
        assert all(i["status"] == 0 for i in info)
    assert np.abs(H.effective(5)).max() < 1e-9 * np.abs(H.effective(4)).max()
    assert np.abs(H.effective(4)).max() > 1e-6
    H.close()


def test_laminate_chain_converges_to_closed_solutions_on_gpu():
    """The three-layer laminate of tests/test_oracle_laminate_hierarchy.py at 512 voxels across:
    the GPU's D_1 .. D_6 along the chain E^11 Y2^o / o! match the closed ODE solutions to the
    second-order discretisation error (about 1e-5 relative at this resolution)."""
    from oracle.hierarchy import multisets
    from paper_1712_05145_gb300 import hom
    from tests.test_oracle_laminate_hierarchy import BOUNDS, LAME, MAX_ORDER, closed_chain
    n = 512
    phase = np.zeros((2, 2, n), dtype=np.uint8)
    phase[:, :, int(BOUNDS[0] * n):int(BOUNDS[1] * n)] = 1
    phase[:, :, int(BOUNDS[1] * n):] = 2
    H = hom.Homogenization(synthetic.Microstructure(phase, LAME, 3.0, 2.0), precision=0)
    for order in range(MAX_ORDER + 1):
        info = H.solve(order, 1e-12)
        assert all(i["status"] == 0 for i in info), order
    ref = closed_chain(MAX_ORDER)
    for o in range(1, MAX_ORDER + 1):
        if o == 1:
            col = 1                                   # load 3A + k, k = y2
        elif o == 2:
            col = 1                                   # load 6A + P, P = Mandel pair (2, 2)
        else:
            col = multisets(o).index((1,) * o)
        got = H.effective(o)[5 if o % 2 == 1 else 0, col]
        assert abs(got - ref[o]) < 5e-5 * abs(ref[o]), (o, got, ref[o])
    H.close()
