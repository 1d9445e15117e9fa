"""GPU parity on two-dimensional cells (N3 = 1) and of order-1 load combinations."""
import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle.hierarchy import Hierarchy
from oracle.lippmann_schwinger import Problem
from oracle.tensors import tensor_to_mandel
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL, TOL_EFF, random_phase, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cell_2d():
    g = (16, 12, 1)
    return synthetic.Microstructure(random_phase(g, 3, 31, p=[0.5, 0.3, 0.2]),
                                    np.array([[1.0, 1.0], [6.0, 4.0], [0.3, 0.2]]), 3.0, 2.0)


@pytest.fixture(scope="module")
def oracle_2d():
    ms = cell_2d()
    h = Hierarchy(Problem(ms.phase, ms.lame, ms.lam0, ms.mu0), tol=1e-12)
    h.order1()      # the paper's alpha = 1 (order 0 here)
    h.order2()      # alpha = 2 (order 1 here)
    return ms, h


@pytest.mark.parametrize("precision", [0, 1])
def test_two_dimensional_cell_matches_oracle(oracle_2d, precision):
    from paper_1712_05145_gb300 import hom
    ms, oh = oracle_2d
    tol = 1e-12 if precision == 0 else 1e-9
    for pass_mode in (1, 2):   # fused plane kernels, split x and y passes
        H = hom.Homogenization(ms, precision=precision, pass_mode=pass_mode)
        for order in (0, 1):
            info = H.solve(order, tol)
            assert all(i["status"] == 0 for i in info), (order, info)
        assert rel_err(H.effective(0), oh.c_eff) < TOL_EFF[precision]
        assert rel_err(H.effective(1), oh.d1) < TOL_EFF[precision] * 10
        tol_f = TOL[precision] * (1 if precision == 0 else 5)
        for L in (0, 4, 16):
            a, k = divmod(L, 3)
            assert rel_err(H.field(1, L), tensor_to_mandel(oh.eps2[(a, k)])) < tol_f, L
        H.close()


def test_two_dimensional_cell_equals_its_extrusion_on_gpu():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.hashin_2d(32)
    ext = synthetic.Microstructure(np.repeat(ms.phase, 2, axis=0), ms.lame, ms.lam0, ms.mu0)
    c = []
    for m in (ms, ext):
        H = hom.Homogenization(m, precision=0)
        info = H.solve(0, 1e-12)
        assert all(i["status"] == 0 for i in info)
        c.append(H.effective(0))
        H.close()
    assert rel_err(c[0], c[1]) < 1e-10


def test_hashin_2d_in_plane_bulk_near_matrix_bulk():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.hashin_2d(128)
    k3, _ = cf.plane_stress_moduli(453.685, 0.3)
    H = hom.Homogenization(ms, precision=1)
    info = H.solve(0, 1e-8, loads=np.array([[1.0, 1.0, 0, 0, 0, 0]]))
    assert info[0]["status"] == 0
    kap = 0.25 * (H.effective(0)[0, 0] + H.effective(0)[1, 0])
    assert abs(kap - k3) / k3 < 0.006          # first-order voxel error of the interfaces
    H.close()


def combos():
    W = np.zeros((3, 18))
    W[0, 0] = W[0, 4] = 1.0            # (grad E)_111 = (grad E)_222 = 1 (Fig. 2 of Sec. 4)
    W[1, 3 * 5 + 1] = 2.0              # E^(12) varying along y2, doubled
    W[2, :] = np.linspace(-1.0, 1.0, 18)
    return W


@pytest.mark.parametrize("precision", [0, 1])
def test_order1_combinations_match_unit_loads(oracle_2d, precision):
    from paper_1712_05145_gb300 import hom
    ms, oh = oracle_2d
    W = combos()
    tol = 1e-12 if precision == 0 else 1e-9
    H = hom.Homogenization(ms, precision=precision)
    H.solve(0, tol)
    info = H.solve(1, tol, loads=W)
    assert len(info) == 3 and all(i["status"] == 0 for i in info)
    d = H.effective(1)
    assert d.shape == (6, 3)
    assert rel_err(d, oh.d1 @ W.T) < TOL_EFF[precision] * 10
    tol_f = TOL[precision] * (1 if precision == 0 else 5)
    for l in range(3):
        ref = sum(W[l, 3 * a + k] * tensor_to_mandel(oh.eps2[(a, k)]) for a in range(6) for k in range(3))
        assert rel_err(H.field(1, l), ref) < tol_f, l
    # order 2 needs the unit loads of order 1
    with pytest.raises(hom.HomError) as e:
        H.solve(2, tol)
    assert e.value.status == hom.HOM_ERR_ORDER
    H.close()


def test_order1_combinations_need_only_their_order0_loads(oracle_2d):
    from paper_1712_05145_gb300 import hom
    ms, oh = oracle_2d
    H = hom.Homogenization(ms, precision=0)
    H.solve(0, 1e-12, loads=np.eye(6)[[1, 0]])      # e22, e11 only, in that order
    W = combos()[:1]
    info = H.solve(1, 1e-12, loads=W)
    assert info[0]["status"] == 0
    assert rel_err(H.effective(1), oh.d1 @ W.T) < TOL_EFF[0] * 10
    with pytest.raises(hom.HomError) as e:
        H.solve(1, 1e-12, loads=combos()[1:2])      # needs e12
    assert e.value.status == hom.HOM_ERR_ORDER
    H.close()


def test_two_dimensional_orders_with_bicgstab(oracle_2d):
    from paper_1712_05145_gb300 import hom
    ms, oh = oracle_2d
    H = hom.Homogenization(ms, precision=0, scheme=hom.HOM_BICGSTAB)
    for order in (0, 1):
        info = H.solve(order, 1e-12)
        assert all(i["status"] == 0 for i in info), (order, info)
    assert rel_err(H.effective(0), oh.c_eff) < TOL_EFF[0]
    assert rel_err(H.effective(1), oh.d1) < TOL_EFF[0] * 10
    H.close()
