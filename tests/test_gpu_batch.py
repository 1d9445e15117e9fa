"""Several RVEs of one grid in one handle (hom_options.n_rve): every launch carries the loads of all
of them, and each RVE's result is bit for bit the one its own handle gives.  hom_set_rve refills a
handle in place."""
import numpy as np
import pytest

from oracle.lippmann_schwinger import Problem
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL, oracle_ls_step_mandel, random_mandel_fields, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rves(grid):
    return [synthetic.random_spheres(grid, seed=31, inclusion_e=10.0),
            synthetic.random_spheres(grid, seed=32, inclusion_e=400.0),
            synthetic.three_phase_spheres(grid, seed=33)]


def solo(ms, precision, tol):
    from paper_1712_05145_gb300 import hom
    H = hom.Homogenization(ms, precision=precision, scheme=hom.HOM_CG)
    info = H.solve(0, tol)
    out = (H.effective(0), [H.field(0, a) for a in (0, 5)], [i["iterations"] for i in info])
    H.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_slots_match_solo_solves_bit_for_bit(precision):
    from paper_1712_05145_gb300 import hom
    grid = (24, 24, 24)
    tol = 1e-10 if precision == 0 else 1e-7
    ms = rves(grid)
    ref = [solo(m, precision, tol) for m in ms]
    H = hom.Homogenization(ms[0], precision=precision, scheme=hom.HOM_CG, n_rve=4)
    for k in (1, 2):
        hom.hom_set_rve(H.h, k, ms[k].phase, ms[k].lame, ms[k].lam0, ms[k].mu0)
    info = H.solve(0, tol, n_loads=18)                  # the first three slots
    assert len(info) == 18 and all(i["status"] == 0 for i in info)
    eff = H.effective(0)
    for k in range(3):
        c, fields, iters = ref[k]
        assert np.array_equal(eff[:, 6 * k:6 * k + 6], c), k
        assert [i["iterations"] for i in info[6 * k:6 * k + 6]] == iters, k
        for a, f in zip((0, 5), fields):
            assert np.array_equal(H.field(0, 6 * k + a), f), (k, a)
    H.close()


def test_set_rve_refills_a_handle_without_allocating():
    from paper_1712_05145_gb300 import hom
    grid = (16, 16, 16)
    a, b = synthetic.random_spheres(grid, seed=41), synthetic.centred_sphere(16, matrix=(0.5, 0.4), inclusion=(30.0, 20.0))
    ref_b = solo(b, hom.HOM_FP32_REFINE, 1e-7)
    H = hom.Homogenization(a, precision=hom.HOM_FP32_REFINE, scheme=hom.HOM_CG)
    H.solve(0, 1e-7)
    before = hom.hom_device_bytes(H.h)
    hom.hom_set_rve(H.h, 0, b.phase, b.lame, b.lam0, b.mu0)
    with pytest.raises(hom.HomError):        # the previous solution was discarded
        H.effective(0)
    H.solve(0, 1e-7)
    assert hom.hom_device_bytes(H.h) == before
    assert np.array_equal(H.effective(0), ref_b[0])
    with pytest.raises(hom.HomError):        # phase values beyond n_phase are refused
        hom.hom_set_rve(H.h, 0, np.full(b.phase.shape, 5, np.uint8), b.lame, b.lam0, b.mu0)
    with pytest.raises(hom.HomError):
        hom.hom_set_rve(H.h, 1, b.phase, b.lame, b.lam0, b.mu0)   # one slot only
    H.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_ls_step_of_each_slot_matches_oracle(precision):
    """hom_ls_apply on a two-slot handle: loads 0-5 use slot 0's RVE, loads 6-11 slot 1's."""
    from paper_1712_05145_gb300 import hom
    grid = (12, 8, 16)
    ms = rves(grid)[:2]
    H = hom.Homogenization(ms[0], precision=precision, n_rve=2)
    hom.hom_set_rve(H.h, 1, ms[1].phase, ms[1].lame, ms[1].lam0, ms[1].mu0)
    eps = random_mandel_fields(12, grid, 5)
    E = np.random.default_rng(9).uniform(-1, 1, size=(12, 6))
    out = torch.empty((12, 6, grid[2], grid[1], grid[0]), dtype=torch.float64, device="cuda")
    hom.hom_ls_apply(H.h, 12, torch.from_numpy(eps).cuda(), E, out)
    got = out.cpu().numpy()
    for k in range(2):
        pb = Problem(ms[k].phase, ms[k].lame, ms[k].lam0, ms[k].mu0)
        ref = np.stack([oracle_ls_step_mandel(pb, eps[6 * k + i], E[6 * k + i]) for i in range(6)])
        assert rel_err(got[6 * k:6 * k + 6], ref) < TOL[precision], k
    H.close()


def test_several_slot_handles_refuse_what_they_do_not_support():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.centred_sphere(8)
    with pytest.raises(hom.HomError):
        hom.Homogenization(ms, scheme=hom.HOM_POLARIZATION, n_rve=2)
    with pytest.raises(hom.HomError):
        hom.Homogenization(ms, n_rve=11)
    H = hom.Homogenization(ms, precision=hom.HOM_FP64, n_rve=2)
    with pytest.raises(hom.HomError):
        H.solve(0, 1e-8, loads=np.eye(6)[:2])
    with pytest.raises(hom.HomError):
        H.solve(0, 1e-8, n_loads=7)
    H.solve(0, 1e-8)
    with pytest.raises(hom.HomError):
        H.solve(1, 1e-8)
    H.close()
