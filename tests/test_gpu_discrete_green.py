"""GPU parity of the rotated finite-difference Green operator (hom_options.green_operator =
HOM_GREEN_ROTATED) against the oracle's RotatedProblem, whose solutions are pinned to a real-space
solve of the same discretisation (tests/test_oracle_discrete_green.py)."""
import numpy as np
import pytest

from oracle import closed_forms
from oracle.discrete_green import RotatedProblem, green_apply_rotated
from oracle import fourier
from oracle.tensors import mandel_to_tensor, tensor_to_mandel, unit_mandel_load
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL, TOL_EFF, TOL_FFT, oracle_ls_step_mandel, random_mandel_fields, random_phase, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRIDS = [(8, 6, 4), (12, 8, 6), (32, 16, 24), (16, 16, 32), (24, 12, 1)]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("grid", GRIDS, ids=["x".join(map(str, g)) for g in GRIDS])
def test_green_contraction_matches_oracle(grid, precision):
    from paper_1712_05145_gb300 import hom
    n1, n2, n3 = grid
    lam0, mu0 = 1.7, 0.9
    rng = np.random.default_rng(3)
    tau = mandel_to_tensor(rng.standard_normal((6, n3, n2, n1)))
    th = fourier.forward(tau)
    ref = tensor_to_mandel(green_apply_rotated(th, grid, lam0, mu0))[..., : n1 // 2 + 1]
    inp = tensor_to_mandel(th)[..., : n1 // 2 + 1]
    ms = synthetic.Microstructure(np.zeros((n3, n2, n1), np.uint8), np.array([[1.0, 1.0]]), lam0, mu0)
    H = hom.Homogenization(ms, precision=precision, green_operator=hom.HOM_GREEN_ROTATED)
    ti = torch.from_numpy(np.stack([inp.real, inp.imag], axis=-1)[None].copy()).cuda()
    to = torch.empty_like(ti)
    hom.hom_green_apply(H.h, 1, ti, to)
    g = to.cpu().numpy()[0]
    assert rel_err(g[..., 0] + 1j * g[..., 1], ref) < TOL_FFT[precision] * 5
    H.close()


@pytest.mark.parametrize("z_mode", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("grid", GRIDS, ids=["x".join(map(str, g)) for g in GRIDS])
def test_ls_step_matches_oracle(grid, precision, z_mode):
    from paper_1712_05145_gb300 import hom
    ms = synthetic.Microstructure(random_phase(grid, 3, 4), np.array([[1.0, 0.5], [12.0, 7.0], [0.2, 0.3]]),
                                  3.0, 2.0)
    pb = RotatedProblem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    eps = random_mandel_fields(2, grid, 8)
    E = np.random.default_rng(2).uniform(-1, 1, size=(2, 6))
    ref = np.stack([oracle_ls_step_mandel(pb, eps[i], E[i]) for i in range(2)])
    H = hom.Homogenization(ms, precision=precision, z_mode=z_mode, green_operator=hom.HOM_GREEN_ROTATED)
    ed = torch.from_numpy(eps).cuda()
    out = torch.empty_like(ed)
    hom.hom_ls_apply(H.h, 2, ed, E, out)
    assert rel_err(out.cpu().numpy(), ref) < TOL[precision]
    H.close()


@pytest.mark.parametrize("scheme", [1, 0])
@pytest.mark.parametrize("precision", [0, 1])
def test_cg_solution_matches_oracle(precision, scheme):
    from paper_1712_05145_gb300 import hom
    if scheme == 0 and precision == 1:
        pytest.skip("the Basic Scheme runs in FP64")
    ms = synthetic.random_spheres((16, 16, 16), seed=5)
    pb = RotatedProblem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    H = hom.Homogenization(ms, precision=precision, scheme=scheme, max_iter=20000,
                           green_operator=hom.HOM_GREEN_ROTATED)
    info = H.solve(0, 1e-12 if precision == 0 else 1e-9)
    assert all(i["status"] == 0 for i in info), info
    for a in (0, 4):
        e, _, _ = pb.cg(pb.rhs(unit_mandel_load(a)), 1e-12)
        assert rel_err(H.field(0, a), tensor_to_mandel(e)) < TOL[precision], a
    _, c_ref = pb.solve_order0(tol=1e-12)
    assert rel_err(H.effective(0), c_ref) < TOL_EFF[precision]
    H.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_laminate_of_odd_thickness_is_exact(precision):
    """5 + 11 layers normal to y1: the rotated operator gives the laminate closed form."""
    from paper_1712_05145_gb300 import hom
    ms = synthetic.laminate((16, 4, 4), split=5)
    exact = closed_forms.laminate_stiffness([tuple(x) for x in ms.lame], ms.volume_fractions())
    H = hom.Homogenization(ms, precision=precision, green_operator=hom.HOM_GREEN_ROTATED)
    H.solve(0, 1e-12 if precision == 0 else 1e-9)
    assert rel_err(H.effective(0), exact) < TOL_EFF[precision]
    H.close()


def test_higher_orders_and_spectral_diagnostics_are_refused():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.centred_sphere(8)
    H = hom.Homogenization(ms, precision=hom.HOM_FP64, green_operator=hom.HOM_GREEN_ROTATED)
    H.solve(0, 1e-10)
    with pytest.raises(hom.HomError):
        H.solve(1, 1e-8)
    with pytest.raises(hom.HomError):
        H.equilibrium_error()
    with pytest.raises(hom.HomError):
        H.field(0, 0, hom.HOM_FIELD_DISPLACEMENT)
    H.close()
