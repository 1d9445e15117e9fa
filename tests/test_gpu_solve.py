"""GPU parity of the order-0 solvers (Basic Scheme, CG, FP32 + FP64 refinement) and C_eff."""
import numpy as np
import pytest

from oracle import closed_forms
from oracle.lippmann_schwinger import Problem
from oracle.tensors import mandel_to_tensor, tensor_to_mandel, unit_mandel_load
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL, TOL_EFF, random_phase, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def oracle_order0(ms, tol=1e-12):
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    sols, c_eff = pb.solve_order0(tol=tol, scheme="cg")
    return [tensor_to_mandel(s) for s in sols], c_eff


@pytest.mark.parametrize("precision,scheme", [(0, 0), (0, 1), (1, 1), (0, 2), (1, 2)])
def test_order0_sphere16_fields_and_ceff(precision, scheme):
    from paper_1712_05145_gb300 import hom
    ms = synthetic.centred_sphere(16)
    ref_f, ref_c = oracle_order0(ms)
    H = hom.Homogenization(ms, precision=precision, scheme=scheme)
    tol = 1e-12 if precision == 0 else 1e-9
    info = H.solve(0, tol)
    assert all(i["status"] == 0 for i in info), info
    assert all(i["rel_residual_fp64"] < tol for i in info), info
    c = H.effective(0)
    assert rel_err(c, ref_c) < TOL_EFF[precision]
    for a in range(6):
        assert rel_err(H.field(0, a), ref_f[a]) < TOL[precision], a
    H.close()


def test_config_c1_sphere32_basic_scheme_fp64():
    """32^3 sphere, f = 0.2, (1,1)/(10,10), C0 = mean, Basic Scheme FP64, E = e11."""
    from paper_1712_05145_gb300 import hom
    ms = synthetic.centred_sphere(32)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    b = pb.rhs(unit_mandel_load(0))
    ref, _, _ = pb.cg(b, 1e-12)
    ref_m = tensor_to_mandel(ref)
    ref_col = pb.mean_stress(ref, unit_mandel_load(0))
    H = hom.Homogenization(ms, precision=hom.HOM_FP64, scheme=hom.HOM_BASIC, max_iter=5000)
    info = H.solve(0, 1e-12, loads=np.eye(6)[:1])
    assert info[0]["status"] == 0 and info[0]["rel_residual_fp64"] < 1e-11
    assert rel_err(H.field(0, 0), ref_m) < 1e-10
    assert rel_err(H.effective(0)[:, 0], ref_col) < 1e-9
    # the configuration's own stopping tolerance
    info = H.solve(0, 1e-8, loads=np.eye(6)[:1])
    assert info[0]["status"] == 0 and 50 < info[0]["iterations"] < 200
    assert rel_err(H.effective(0)[:, 0], ref_col) < 1e-6
    H.close()


@pytest.mark.parametrize("precision,scheme", [(0, 0), (0, 1), (1, 1), (0, 2), (1, 2)])
def test_config_c1_laminate32_closed_form(precision, scheme):
    from paper_1712_05145_gb300 import hom
    ms = synthetic.laminate((32, 32, 32))
    exact = closed_forms.laminate_stiffness([tuple(ms.lame[0]), tuple(ms.lame[1])], [0.5, 0.5])
    H = hom.Homogenization(ms, precision=precision, scheme=scheme)
    info = H.solve(0, 1e-10 if precision == 0 else 1e-9)
    assert all(i["status"] == 0 for i in info), info
    assert rel_err(H.effective(0), exact) < (1e-9 if precision == 0 else 1e-6)
    H.close()


@pytest.mark.parametrize("pass_mode", [0, 2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_random_spheres_32_cg_vs_oracle(precision, pass_mode):
    """Fused plane kernels (0), split x and y passes (2), cluster plane passes (3, FP32)."""
    from paper_1712_05145_gb300 import hom
    ms = synthetic.random_spheres((32, 32, 32), seed=3)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    loads = [0, 3]
    refs = []
    for a in loads:
        e, _, _ = pb.cg(pb.rhs(unit_mandel_load(a)), 1e-12)
        refs.append(tensor_to_mandel(e))
    H = hom.Homogenization(ms, precision=precision, scheme=hom.HOM_CG, pass_mode=pass_mode)
    info = H.solve(0, 1e-12 if precision == 0 else 1e-9)
    assert all(i["status"] == 0 for i in info), info
    for r, a in zip(refs, loads):
        assert rel_err(H.field(0, a), r) < TOL[precision]
    c = H.effective(0)
    assert rel_err(c, c.T) < (1e-9 if precision == 0 else 1e-6)
    H.close()


def test_homogeneous_medium_gives_zero_strain():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.centred_sphere(8, matrix=(2.0, 3.0), inclusion=(2.0, 3.0))
    for prec, scheme in [(0, 0), (1, 1)]:
        H = hom.Homogenization(ms, precision=prec, scheme=scheme)
        info = H.solve(0, 1e-8)
        assert all(i["status"] == 0 for i in info)
        assert np.abs(H.field(0, 2)).max() < 1e-12
        expect = np.diag([6.0] * 6) + 2.0 * (np.arange(6)[:, None] < 3) * (np.arange(6)[None] < 3)
        np.testing.assert_allclose(H.effective(0), expect, atol=1e-10)
        H.close()


def test_custom_loads_are_linear_combinations():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.Microstructure(random_phase((16, 8, 12), 3, 4), np.array([[1.0, 1.0], [5.0, 2.0], [0.5, 0.4]]),
                                  2.0, 1.5)
    H = hom.Homogenization(ms, precision=0)
    H.solve(0, 1e-12)
    c = H.effective(0)
    L = np.random.default_rng(2).standard_normal((4, 6))
    H.solve(0, 1e-12, loads=L)
    np.testing.assert_allclose(H.effective(0), c @ L.T, atol=1e-9 * np.abs(c).max())
    H.close()


def test_not_converged_is_reported():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.random_spheres((16, 16, 16), seed=2)
    H = hom.Homogenization(ms, precision=0, scheme=hom.HOM_CG, max_iter=3, check_every=1, max_refine=0)
    info = H.solve(0, 1e-12)
    assert all(i["status"] == hom.HOM_ERR_NOT_CONVERGED for i in info)
    assert all(i["iterations"] <= 3 for i in info)
    H.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_bicgstab_high_contrast_three_phases(precision):
    """BiCGSTAB (the paper's Krylov solver) reaches the oracle's discrete solution on a
    three-phase cell with a soft and a stiff phase (contrast 100 each way)."""
    from paper_1712_05145_gb300 import hom
    g = (16, 12, 8)
    ms = synthetic.Microstructure(random_phase(g, 3, 41, p=[0.5, 0.3, 0.2]),
                                  np.array([[1.0, 1.0], [1e2, 1e2], [1e-2, 1e-2]]), 50.0, 50.0)
    ref_f, ref_c = oracle_order0(ms)
    H = hom.Homogenization(ms, precision=precision, scheme=hom.HOM_BICGSTAB, max_iter=5000)
    tol = 1e-11 if precision == 0 else 1e-8
    info = H.solve(0, tol)
    assert all(i["status"] == 0 for i in info), info
    assert rel_err(H.effective(0), ref_c) < (1e-8 if precision == 0 else 1e-5)
    for a in (0, 5):
        assert rel_err(H.field(0, a), ref_f[a]) < (1e-8 if precision == 0 else 1e-4), a
    H.close()


@pytest.mark.parametrize("precision,scheme", [(0, 1), (1, 1), (0, 2), (0, 0)])
def test_zero_load_is_exact_and_free(precision, scheme):
    """A zero macroscopic strain has b = 0: the solution 0 is exact, with no iteration."""
    from paper_1712_05145_gb300 import hom
    ms = synthetic.random_spheres((16, 16, 16), seed=9)
    H = hom.Homogenization(ms, precision=precision, scheme=scheme)
    loads = np.zeros((2, 6))
    loads[1, 0] = 1.0
    info = H.solve(0, 1e-8, loads=loads)
    assert info[0]["status"] == 0 and info[0]["iterations"] <= (1 if scheme == 0 else 0)
    assert np.abs(H.field(0, 0)).max() == 0.0
    assert np.abs(H.effective(0)[:, 0]).max() == 0.0
    assert info[1]["status"] == 0 and info[1]["iterations"] > 0
    H.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_launch_shape_gives_identical_results(precision):
    """The autotuner changes loads per launch, tile widths and which z-stage kernel runs.  Loads
    per launch and tile widths keep every per-load reduction in its order, so with the same z
    kernel the solution is the same bits (the cluster z pass's two copy forms, per-element and
    TMA, run the same arithmetic); a different z kernel (cluster or single CTA) computes the same
    contraction in another compiled kernel, so there the results agree within the parity
    tolerance."""
    from paper_1712_05145_gb300 import hom
    ms = synthetic.random_spheres((32, 32, 32), seed=12)
    out = []
    for tune in (0, 1):
        H = hom.Homogenization(ms, precision=precision, autotune=tune)
        info = H.solve(0, 1e-8)
        assert all(i["status"] == 0 for i in info)
        chunk, lg = hom.hom_launch_config(H.h)
        cluster, zlg = hom.hom_zpass_config(H.h)
        assert chunk >= 1
        if tune:   # the tuner reports its choice: a single-CTA tile width or a cluster tile width
            assert (cluster == 0 and lg >= 0) or (cluster in (1, 2) and zlg >= 0)
        else:      # the cluster z pass, in its TMA form for FP32 transforms (32 x 17 columns: even)
            assert lg == -1 and cluster == (2 if precision == 1 else 1)
        out.append((H.effective(0), H.field(0, 2), cluster))
        H.close()
    if (out[0][2] > 0) == (out[1][2] > 0):
        assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    else:
        assert rel_err(out[1][0], out[0][0]) < TOL_EFF[precision]
        assert rel_err(out[1][1], out[0][1]) < TOL[precision]


def test_fp32_mode_residual_certified_at_1e10():
    """The FP32 mode's FP64 passes (double-float arithmetic) certify a residual of 1e-10: the
    oracle recomputes the literal residual of the GPU solution and agrees with the reported one."""
    from paper_1712_05145_gb300 import hom
    ms = synthetic.random_spheres((24, 24, 24), seed=5, inclusion_e=100.0)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    H = hom.Homogenization(ms, precision=hom.HOM_FP32_REFINE, max_refine=12)
    info = H.solve(0, 1e-10, loads=np.eye(6)[[0, 3]])
    assert all(i["status"] == 0 for i in info), info
    for k, a in enumerate((0, 3)):
        res = pb.residual(mandel_to_tensor(H.field(0, k)), pb.rhs(unit_mandel_load(a)))
        assert res < 1e-10, (a, res)
        assert abs(res - info[k]["rel_residual_fp64"]) < 0.05 * res + 1e-13, (res, info[k])
    H.close()


def test_tuning_cache_reuses_the_tuned_shape(tmp_path, monkeypatch):
    """With HOM_TUNE_CACHE set, the first autotuned handle of a grid writes its launch shape and a
    second handle of the same grid and options reads it back instead of timing again."""
    from paper_1712_05145_gb300 import hom
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("HOM_TUNE_CACHE", str(path))
    ms = synthetic.random_spheres((32, 32, 32), seed=12)
    shapes, effs = [], []
    for _ in range(2):
        H = hom.Homogenization(ms, precision=hom.HOM_FP32_REFINE, autotune=1)
        H.solve(0, 1e-7)
        shapes.append((hom.hom_launch_config(H.h), hom.hom_zpass_config(H.h), hom.hom_plane_config(H.h)))
        effs.append(H.effective(0))
        H.close()
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and "|" in lines[0]
    assert shapes[0] == shapes[1]
    assert np.array_equal(effs[0], effs[1])
