"""TMA tile copies in the split y pass (hom_options.y_mode 0 and 1) and the cluster z pass (z_mode 0
and 2), FP32 transforms, against the per-element copies (y_mode 2, z_mode 3).

The z stage of the LS step (Sec. 2: the transform along z, eta_hat = -Gamma0_hat(xi) : tau_hat with
eta_hat(0) = 0, the inverse transform) runs the same arithmetic as the plain cluster z pass, with
each CTA's tile moved by tensor loads and stores.  Cases: oracle parity on grids whose z columns
take two boxes (N3 = 384, 512) and whose last tile is ragged (the plane's spectrum columns are not
a multiple of the tile width); bit-identical results against the plain cluster z pass with the
same tile width, for one LS step and a whole solve; the fallback where a plane has an odd number
of spectrum columns (16-byte tensor strides impossible).  The y pass (the y-axis FFT of column tiles
of one z-plane, with the packed x = 0 / Nyquist columns separated or packed) is checked the same
way on split grids, with y lengths whose columns take two boxes (N2 = 384, 512).
"""
import numpy as np
import pytest

from oracle.lippmann_schwinger import Problem
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL, oracle_ls_step_mandel, random_mandel_fields, random_phase, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAME = np.array([[1.0, 1.0], [8.0, 5.0], [0.4, 0.3]])


def _ms(grid, seed):
    return synthetic.Microstructure(random_phase(grid, 3, seed, p=[0.5, 0.3, 0.2]), LAME, 4.0, 2.5)


def _config(H):
    from paper_1712_05145_gb300 import hom
    return hom.hom_zpass_config(H.h)


# (grid, expected z stage): plane_c = n2 (n1/2 + 1); N3 = 384 and 512 take two boxes of 192 / 256
# z-planes; 312, 54 and 108 spectrum columns leave a ragged last tile of the default width (16
# columns at N3 = 384 and 512, 64 at N3 = 64); 15 columns (odd) rule the TMA form out
GRIDS = [((24, 24, 384), 2), ((16, 6, 512), 2), ((16, 12, 64), 2), ((8, 3, 32), 1)]


@pytest.mark.parametrize("grid,kind", GRIDS, ids=["x".join(map(str, g[0])) for g in GRIDS])
def test_ls_step_matches_oracle_and_plain_cluster_bits(grid, kind):
    from paper_1712_05145_gb300 import hom
    ms = _ms(grid, sum(grid))
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    nrhs = 2
    eps = random_mandel_fields(nrhs, ms.grid, 7)
    E = np.random.default_rng(9).uniform(-1, 1, size=(nrhs, 6))
    ref = np.stack([oracle_ls_step_mandel(pb, eps[i], E[i]) for i in range(nrhs)])
    outs = {}
    for z_mode in (2, 3, 0):
        H = hom.Homogenization(ms, precision=1, z_mode=z_mode)
        cluster, lg = _config(H)
        assert cluster == (1 if z_mode == 3 else kind), (z_mode, cluster, lg)
        ed = torch.from_numpy(eps).cuda()
        out = torch.empty_like(ed)
        hom.hom_ls_apply(H.h, nrhs, ed, E, out)
        outs[z_mode] = out.cpu().numpy()
        H.close()
    assert rel_err(outs[2], ref) < TOL[1]
    # same tile width, same FFT and contraction code: the same bits
    assert np.array_equal(outs[2], outs[3])
    assert np.array_equal(outs[0], outs[2])


def test_solve_bits_and_autotuned_width():
    """A whole FP32 + refinement solve with the TMA form gives the C_eff and fields of the plain
    cluster z pass bit for bit; with autotuning, z_mode 2 keeps the TMA form and tunes its width."""
    from paper_1712_05145_gb300 import hom
    ms = _ms((32, 24, 128), 4)
    loads = np.eye(6)
    res = {}
    for z_mode in (2, 3):
        H = hom.Homogenization(ms, precision=1, z_mode=z_mode)
        info = H.solve(0, 1e-6, loads=loads)
        assert all(i["status"] == 0 for i in info), info
        res[z_mode] = (H.effective(0), np.stack([H.field(0, k) for k in range(6)]))
        H.close()
    assert np.array_equal(res[2][0], res[3][0])
    assert np.array_equal(res[2][1], res[3][1])
    H = hom.Homogenization(ms, precision=1, z_mode=2, autotune=1)
    info = H.solve(0, 1e-6, loads=loads)
    assert all(i["status"] == 0 for i in info), info
    cluster, lg = _config(H)
    assert cluster == 2 and 1 <= lg <= 6, (cluster, lg)
    assert rel_err(H.effective(0), res[3][0]) < 1e-5
    H.close()


def test_fp64_mode_ignores_the_tma_form():
    """z_mode 2 on an FP64 handle runs the plain cluster z pass (the TMA form is FP32 only)."""
    from paper_1712_05145_gb300 import hom
    ms = _ms((16, 12, 64), 3)
    H = hom.Homogenization(ms, precision=0, z_mode=2)
    assert _config(H)[0] == 1
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    eps = random_mandel_fields(1, ms.grid, 2)
    E = np.random.default_rng(1).uniform(-1, 1, size=(1, 6))
    ed = torch.from_numpy(eps).cuda()
    out = torch.empty_like(ed)
    hom.hom_ls_apply(H.h, 1, ed, E, out)
    assert rel_err(out.cpu().numpy(), oracle_ls_step_mandel(pb, eps[0], E[0])[None]) < TOL[0]
    H.close()


def _yconfig(H):
    from paper_1712_05145_gb300 import hom
    return hom.hom_ypass_config(H.h)


# (grid, TMA expected): split x and y passes (pass_mode 2); h = N1/2 and plane_c = N2 (h + 1) must be
# even; N2 = 384 and 512 take two boxes of 192 / 256 rows
YGRIDS = [((16, 12, 8), 1), ((8, 384, 2), 1), ((16, 512, 2), 1), ((32, 24, 16), 1), ((6, 12, 4), 0),
          ((8, 3, 4), 0)]


@pytest.mark.parametrize("grid,tma", YGRIDS, ids=["x".join(map(str, g[0])) for g in YGRIDS])
def test_y_pass_ls_step_matches_oracle_and_plain_bits(grid, tma):
    from paper_1712_05145_gb300 import hom
    ms = _ms(grid, 3 * sum(grid))
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    nrhs = 2
    eps = random_mandel_fields(nrhs, ms.grid, 17)
    E = np.random.default_rng(19).uniform(-1, 1, size=(nrhs, 6))
    ref = np.stack([oracle_ls_step_mandel(pb, eps[i], E[i]) for i in range(nrhs)])
    outs = {}
    for y_mode in (1, 2, 0):
        H = hom.Homogenization(ms, precision=1, pass_mode=2, y_mode=y_mode)
        lg, used = _yconfig(H)
        assert lg >= 0
        assert used == (0 if y_mode == 2 else tma), (y_mode, lg, used)
        ed = torch.from_numpy(eps).cuda()
        out = torch.empty_like(ed)
        hom.hom_ls_apply(H.h, nrhs, ed, E, out)
        outs[y_mode] = out.cpu().numpy()
        H.close()
    assert rel_err(outs[1], ref) < TOL[1]
    assert np.array_equal(outs[1], outs[2])
    assert np.array_equal(outs[0], outs[1])


def test_y_and_z_tma_solve_bits_and_autotune():
    """Both TMA forms at once through a whole FP32 + refinement solve on a split grid equal the
    per-element copies bit for bit; autotuning with y_mode 1 keeps the TMA y pass."""
    from paper_1712_05145_gb300 import hom
    ms = _ms((64, 48, 32), 6)
    loads = np.eye(6)[[0, 2, 4]]
    res = {}
    for modes in ((1, 2), (2, 3)):
        H = hom.Homogenization(ms, precision=1, pass_mode=2, y_mode=modes[0], z_mode=modes[1])
        assert _yconfig(H)[1] == (1 if modes[0] == 1 else 0)
        assert _config(H)[0] == (2 if modes[1] == 2 else 1)
        info = H.solve(0, 1e-6, loads=loads)
        assert all(i["status"] == 0 for i in info), info
        res[modes] = (H.effective(0), np.stack([H.field(0, k) for k in range(3)]))
        H.close()
    assert np.array_equal(res[(1, 2)][0], res[(2, 3)][0])
    assert np.array_equal(res[(1, 2)][1], res[(2, 3)][1])
    H = hom.Homogenization(ms, precision=1, pass_mode=2, y_mode=1, autotune=1)
    info = H.solve(0, 1e-6, loads=loads)
    assert all(i["status"] == 0 for i in info), info
    assert _yconfig(H)[1] == 1
    H.close()
