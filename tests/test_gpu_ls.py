"""GPU parity of one Lippmann-Schwinger step (steps a1-a5 of the hot path) against the oracle."""
import numpy as np
import pytest

from oracle.lippmann_schwinger import Problem
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL, oracle_ls_step_mandel, random_mandel_fields, random_phase, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cases():
    yield "sphere8", synthetic.centred_sphere(8)
    yield "laminate", synthetic.laminate((16, 8, 8), split=5)
    g = (12, 6, 4)
    yield "random3", synthetic.Microstructure(random_phase(g, 3, 1), np.array([[1.0, 0.5], [10.0, 4.0], [0.2, 0.3]]),
                                              2.0, 1.5)
    yield "sphere32", synthetic.centred_sphere(32)
    g = (32, 64, 16)
    yield "aniso", synthetic.Microstructure(random_phase(g, 2, 2), np.array([[1.0, 1.0], [50.0, 30.0]]), 20.0, 12.0)
    yield "odd_h", synthetic.Microstructure(random_phase((6, 12, 9 if False else 12), 2, 3),
                                            np.array([[1.0, 1.0], [3.0, 2.0]]), 2.0, 1.5)


CASES = list(cases())


@pytest.mark.parametrize("z_mode", [0, 1, 3])
@pytest.mark.parametrize("pass_mode", [0, 2, 3])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,ms", CASES, ids=[c[0] for c in CASES])
def test_ls_step_matches_oracle(name, ms, precision, pass_mode, z_mode):
    """Fused plane kernels (pass_mode 0 on these grids), split x / y passes (pass_mode 2) and
    cluster plane passes (pass_mode 3, FP32 transforms); the cluster z pass (z_mode 0, on grids
    with N3 >= 16; TMA tile copies for FP32 transforms where they fit), the single-CTA z pass
    (z_mode 1) and the cluster z pass with per-element copies (z_mode 3)."""
    from paper_1712_05145_gb300 import hom
    if pass_mode == 3 and precision == 1 and (ms.grid[0] // 2) % 2:
        with pytest.raises(hom.HomError):   # no cluster of 2, 4 or 8 divides an odd N1/2
            hom.Homogenization(ms, precision=precision, pass_mode=pass_mode)
        return
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    nrhs = 3
    eps = random_mandel_fields(nrhs, ms.grid, 11)
    rng = np.random.default_rng(5)
    E = rng.uniform(-1, 1, size=(nrhs, 6))
    ref = np.stack([oracle_ls_step_mandel(pb, eps[i], E[i]) for i in range(nrhs)])
    H = hom.Homogenization(ms, precision=precision, pass_mode=pass_mode, z_mode=z_mode)
    ed = torch.from_numpy(eps).cuda()
    out = torch.empty_like(ed)
    hom.hom_ls_apply(H.h, nrhs, ed, E, out)
    assert rel_err(out.cpu().numpy(), ref) < TOL[precision]
    # zero strain input: the right-hand side b = -Gamma0 * (C : E)
    hom.hom_ls_apply(H.h, nrhs, None, E, out)
    ref0 = np.stack([oracle_ls_step_mandel(pb, 0 * eps[i], E[i]) for i in range(nrhs)])
    assert rel_err(out.cpu().numpy(), ref0) < TOL[precision]
    H.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_ls_step_chunking_gives_identical_results(precision):
    """Spectra transformed one load per launch or all loads per launch: same bits."""
    from paper_1712_05145_gb300 import hom
    ms = synthetic.centred_sphere(16)
    eps = torch.from_numpy(random_mandel_fields(5, ms.grid, 3)).cuda()
    E = np.random.default_rng(1).uniform(-1, 1, size=(5, 6))
    outs = []
    for chunk in (1, 2, 5):
        H = hom.Homogenization(ms, precision=precision, rhs_chunk=chunk)
        o = torch.empty_like(eps)
        hom.hom_ls_apply(H.h, 5, eps, E, o)
        outs.append(o.cpu().numpy())
        H.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("precision", [0, 1])
def test_plane_larger_than_one_cta_uses_split_passes(precision):
    """256 x 128 x 8: (N1/2) * N2 = 16384 complex values per plane, too many for one CTA."""
    from paper_1712_05145_gb300 import hom
    grid = (256, 128, 8)
    ms = synthetic.Microstructure(random_phase(grid, 2, 9), np.array([[1.0, 1.0], [20.0, 12.0]]), 10.0, 6.0)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    eps = random_mandel_fields(1, grid, 12)
    E = np.array([[0.3, -0.2, 0.1, 0.5, 0.0, -0.4]])
    ref = oracle_ls_step_mandel(pb, eps[0], E[0])
    with pytest.raises(hom.HomError):
        hom.Homogenization(ms, precision=precision, pass_mode=1)
    H = hom.Homogenization(ms, precision=precision)
    ed = torch.from_numpy(eps).cuda()
    out = torch.empty_like(ed)
    hom.hom_ls_apply(H.h, 1, ed, E, out)
    assert rel_err(out.cpu().numpy()[0], ref) < TOL[precision]
    H.close()


@pytest.fixture(scope="module")
def deep_grid_case():
    from oracle.tensors import tensor_to_mandel, unit_mandel_load
    g = (8, 6, 512)
    ms = synthetic.Microstructure(random_phase(g, 3, 8, p=[0.5, 0.3, 0.2]),
                                  np.array([[1.0, 1.0], [8.0, 5.0], [0.4, 0.3]]), 4.0, 2.5)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    eps = random_mandel_fields(2, ms.grid, 21)
    E = np.random.default_rng(3).uniform(-1, 1, size=(2, 6))
    ref = np.stack([oracle_ls_step_mandel(pb, eps[i], E[i]) for i in range(2)])
    sols = [tensor_to_mandel(pb.cg(pb.rhs(unit_mandel_load(a)), 1e-12)[0]) for a in (0, 5)]
    return ms, eps, E, ref, sols


@pytest.mark.parametrize("z_mode", [0, 1, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_split_z_stage_on_deep_grid(deep_grid_case, precision, z_mode):
    """N3 = 512: with the single-CTA z pass (z_mode 1) the fused z tiles would be narrower than a
    sector, so the z stage runs as per-component z FFTs and a pointwise contraction; the cluster z
    pass (z_mode 0 in its TMA form for FP32, z_mode 3 with per-element copies) keeps it one pass.
    LS step and solve against the oracle."""
    from paper_1712_05145_gb300 import hom
    ms, eps, E, ref, sols = deep_grid_case
    H = hom.Homogenization(ms, precision=precision, z_mode=z_mode)
    ed = torch.from_numpy(eps).cuda()
    out = torch.empty_like(ed)
    hom.hom_ls_apply(H.h, 2, ed, E, out)
    assert rel_err(out.cpu().numpy(), ref) < TOL[precision]
    tol = 1e-12 if precision == 0 else 1e-8
    info = H.solve(0, tol, loads=np.eye(6)[[0, 5]])
    assert all(i["status"] == 0 for i in info), info
    for k in range(2):
        assert rel_err(H.field(0, k), sols[k]) < (1e-10 if precision == 0 else 1e-5), k
    H.close()
