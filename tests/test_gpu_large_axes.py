"""GPU parity at the axis lengths of the largest workload (512^3) and its neighbours.

The transforms of 512-point and 384-point axes use their own radix sequences and, for x-y planes
above one CTA's shared memory, the split x and y passes.  These cases compare them element by
element with the oracle's FFT (its radix-2 recursion, and the DFT matrix on axes with a factor 3)
and one Lippmann-Schwinger step (Sec. 2, Eq. auxiliary_problem and the Green operator) on grids
that reach every one of those lengths on each axis while the oracle still finishes in seconds.
"""
import numpy as np
import pytest

from oracle import fourier
from oracle.lippmann_schwinger import Problem
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL, TOL_FFT, oracle_ls_step_mandel, random_mandel_fields, random_phase, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# x half-lengths 256 / 192 / 96, y lengths 512 / 384 / 256 / 192, z lengths 512 / 384 / 256 / 192
FFT_GRIDS = [(512, 512, 2), (384, 256, 2), (8, 192, 4), (8, 384, 2), (512, 8, 4),
             (4, 6, 512), (4, 8, 384), (6, 4, 256), (4, 4, 192)]


def _uniform(grid, precision, **kw):
    from paper_1712_05145_gb300 import hom
    n1, n2, n3 = grid
    ms = synthetic.Microstructure(np.zeros((n3, n2, n1), np.uint8), np.array([[1.0, 1.0]]), 1.0, 1.0)
    return hom.Homogenization(ms, precision=precision, **kw)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("grid", FFT_GRIDS, ids=["x".join(map(str, g)) for g in FFT_GRIDS])
def test_fft_at_large_axis_lengths_matches_oracle(grid, precision):
    from paper_1712_05145_gb300 import hom
    n1, n2, n3 = grid
    rng = np.random.default_rng(sum(grid))
    nf = 2
    f = rng.standard_normal((nf, n3, n2, n1))
    ref = (fourier.forward(f) * (n1 * n2 * n3))[..., : n1 // 2 + 1]
    H = _uniform(grid, precision)
    fd = torch.from_numpy(f).cuda()
    out = torch.empty((nf, n3, n2, n1 // 2 + 1, 2), dtype=torch.float64, device="cuda")
    hom.hom_fft_forward(H.h, nf, fd, out)
    got = out.cpu().numpy()
    assert rel_err(got[..., 0] + 1j * got[..., 1], ref) < TOL_FFT[precision]
    back = torch.empty_like(fd)
    hom.hom_fft_inverse(H.h, nf, out, back)
    assert rel_err(back.cpu().numpy() / (n1 * n2 * n3), f) < TOL_FFT[precision]
    H.close()


LS_GRIDS = [(512, 256, 2), (256, 512, 2), (384, 384, 2), (8, 8, 512)]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("grid", LS_GRIDS, ids=["x".join(map(str, g)) for g in LS_GRIDS])
def test_ls_step_at_large_axis_lengths_matches_oracle(grid, precision):
    from paper_1712_05145_gb300 import hom
    ms = synthetic.Microstructure(random_phase(grid, 3, 9), np.array([[1.0, 0.5], [30.0, 12.0], [0.3, 0.2]]),
                                  8.0, 4.0)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    nrhs = 2
    eps = random_mandel_fields(nrhs, grid, 21)
    E = np.random.default_rng(6).uniform(-1, 1, size=(nrhs, 6))
    ref = np.stack([oracle_ls_step_mandel(pb, eps[i], E[i]) for i in range(nrhs)])
    H = hom.Homogenization(ms, precision=precision)
    ed = torch.from_numpy(eps).cuda()
    out = torch.empty_like(ed)
    hom.hom_ls_apply(H.h, nrhs, ed, E, out)
    assert rel_err(out.cpu().numpy(), ref) < TOL[precision]
    H.close()
