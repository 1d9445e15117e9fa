"""GPU parity of the transforms (steps a2, a4) and of the Green contraction (a3)."""
import numpy as np
import pytest

from oracle import fourier
from oracle.lippmann_schwinger import green_apply
from oracle.tensors import mandel_to_tensor, tensor_to_mandel
from paper_1712_05145_gb300 import synthetic
from tests.helpers import TOL_FFT, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRIDS = [(8, 6, 4), (6, 4, 3), (12, 8, 6), (32, 32, 32), (16, 48, 24), (64, 16, 8), (24, 12, 96), (128, 64, 8)]


def make(grid, precision):
    from paper_1712_05145_gb300 import hom
    n1, n2, n3 = grid
    ms = synthetic.Microstructure(np.zeros((n3, n2, n1), np.uint8), np.array([[1.0, 1.0]]), 1.0, 1.0)
    return hom.Homogenization(ms, precision=precision)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("grid", GRIDS)
def test_fft_forward_and_inverse_match_oracle(grid, precision):
    from paper_1712_05145_gb300 import hom
    n1, n2, n3 = grid
    rng = np.random.default_rng(hash(grid) % 1000)
    nf = 3
    f = rng.standard_normal((nf, n3, n2, n1))
    ref = fourier.forward(f) * (n1 * n2 * n3)
    ref = ref[..., : n1 // 2 + 1]
    H = make(grid, precision)
    fd = torch.from_numpy(f).cuda()
    out = torch.empty((nf, n3, n2, n1 // 2 + 1, 2), dtype=torch.float64, device="cuda")
    hom.hom_fft_forward(H.h, nf, fd, out)
    got = out.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    assert rel_err(got, ref) < TOL_FFT[precision]
    back = torch.empty_like(fd)
    hom.hom_fft_inverse(H.h, nf, out, back)
    assert rel_err(back.cpu().numpy() / (n1 * n2 * n3), f) < TOL_FFT[precision]
    H.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("grid,lam0,mu0", [((8, 6, 4), 5.5, 5.5), ((12, 12, 12), 0.0, 1.0),
                                           ((32, 16, 24), -0.3, 2.0), ((16, 16, 16), 2.5, 0.7)])
def test_green_contraction_matches_oracle(grid, lam0, mu0, precision):
    from paper_1712_05145_gb300 import hom
    n1, n2, n3 = grid
    rng = np.random.default_rng(7)
    tau = mandel_to_tensor(rng.standard_normal((6, n3, n2, n1)))
    th = fourier.forward(tau)                                       # Hermitian coefficients
    eta = green_apply(th, grid, lam0, mu0)
    ref = tensor_to_mandel(eta)[..., : n1 // 2 + 1]
    inp = tensor_to_mandel(th)[..., : n1 // 2 + 1]
    ms = synthetic.Microstructure(np.zeros((n3, n2, n1), np.uint8), np.array([[1.0, 1.0]]), lam0, mu0)
    H = hom.Homogenization(ms, precision=precision)
    ti = torch.from_numpy(np.stack([inp.real, inp.imag], axis=-1)[None].copy()).cuda()
    to = torch.empty_like(ti)
    hom.hom_green_apply(H.h, 1, ti, to)
    g = to.cpu().numpy()[0]
    assert rel_err(g[..., 0] + 1j * g[..., 1], ref) < TOL_FFT[precision] * 5
    H.close()
