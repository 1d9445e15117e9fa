"""The allocation-free Lippmann-Schwinger step agrees with the handle-based one.

hom_ls_apply_noalloc serves callers that cannot allocate device memory: it keeps its scratch
in a fixed device array inside the library.  This file is collected last on purpose, so that
a run stopping at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1712_05145_gb300 import synthetic
from tests.helpers import random_mandel_fields, random_phase

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(None if t is None else t.data_ptr())


def _noalloc(lib, grid, phase_dev, lame, lam0, mu0, nrhs, eps_in, E, out, stream):
    g = (ctypes.c_int32 * 3)(*grid)
    lame = np.ascontiguousarray(lame, dtype=np.float64)
    E_p = None if E is None else np.ascontiguousarray(E, dtype=np.float64)
    fn = lib.hom_ls_apply_noalloc
    fn.restype = ctypes.c_int32
    fn.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                   ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn(g, ctypes.c_void_p(phase_dev.data_ptr()), lame.shape[0], ctypes.c_void_p(lame.ctypes.data),
              lam0, mu0, nrhs, _ptr(eps_in), ctypes.c_void_p(None if E_p is None else E_p.ctypes.data),
              _ptr(out), ctypes.c_void_p(stream))


def _case(grid, nrhs):
    ms = synthetic.Microstructure(random_phase(grid, 3, 31), np.array([[1.0, 1.0], [8.0, 5.0], [0.4, 0.3]]),
                                  3.0, 2.0)
    eps = torch.from_numpy(random_mandel_fields(nrhs, grid, 17)).cuda()
    E = np.random.default_rng(4).uniform(-1, 1, size=(nrhs, 6))
    return ms, eps, E


def _reference(ms, nrhs, eps, E):
    from paper_1712_05145_gb300 import hom
    H = hom.Homogenization(ms, precision=hom.HOM_FP64)
    ref = torch.empty((nrhs, 6) + tuple(ms.phase.shape), dtype=torch.float64, device="cuda")
    hom.hom_ls_apply(H.h, nrhs, eps, E, ref)
    torch.cuda.synchronize()
    H.close()
    return ref


def _err(out, ref):
    scale = max(ref.abs().max().item(), 1e-300)
    return (out - ref).abs().max().item() / scale


@pytest.mark.parametrize("grid", [(32, 24, 16), (64, 64, 64), (32, 16, 1)])
@pytest.mark.parametrize("with_eps,with_E", [(True, True), (False, True), (True, False)])
def test_noalloc_step_matches_ls_apply_on_two_calls(grid, with_eps, with_E):
    from paper_1712_05145_gb300 import hom
    lib = hom.load_library()
    lib.hom_noalloc_last_error.restype = ctypes.c_char_p
    nrhs = 2 if grid[2] > 32 else 3
    ms, eps, E = _case(grid, nrhs)
    eps_in = eps if with_eps else None
    E_in = E if with_E else None
    ref = _reference(ms, nrhs, eps_in, E_in)
    phase_dev = torch.from_numpy(ms.phase).cuda()
    side = torch.cuda.Stream()   # a stream other than the current one
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        torch.cuda.synchronize()
        s = _noalloc(lib, grid, phase_dev, ms.lame, ms.lam0, ms.mu0, nrhs, eps_in, E_in, out, side.cuda_stream)
        assert s == hom.HOM_OK, lib.hom_noalloc_last_error()
        side.synchronize()
        assert _err(out, ref) < 1e-12


def test_noalloc_in_place_matches_ls_apply():
    from paper_1712_05145_gb300 import hom
    lib = hom.load_library()
    lib.hom_noalloc_last_error.restype = ctypes.c_char_p
    grid, nrhs = (32, 24, 16), 2
    ms, eps, E = _case(grid, nrhs)
    ref = _reference(ms, nrhs, eps, E)
    phase_dev = torch.from_numpy(ms.phase).cuda()
    buf = eps.clone()
    s = _noalloc(lib, grid, phase_dev, ms.lame, ms.lam0, ms.mu0, nrhs, buf, E, buf,
                 torch.cuda.current_stream().cuda_stream)
    assert s == hom.HOM_OK, lib.hom_noalloc_last_error()
    torch.cuda.synchronize()
    assert _err(buf, ref) < 1e-12


def test_noalloc_phase_values_past_the_table_stay_in_bounds():
    """Phase bytes >= n_phase read a zero row of the padded table: no CUDA error, finite output."""
    from paper_1712_05145_gb300 import hom
    lib = hom.load_library()
    lib.hom_noalloc_last_error.restype = ctypes.c_char_p
    grid, nrhs = (32, 24, 16), 1
    ms, eps, E = _case(grid, nrhs)
    phase = ms.phase.copy()
    phase[0, 0, :4] = [2, 3, 200, 255]        # n_phase is 3
    phase_dev = torch.from_numpy(phase).cuda()
    out = torch.empty_like(eps)
    s = _noalloc(lib, grid, phase_dev, ms.lame, ms.lam0, ms.mu0, nrhs, eps, E, out,
                 torch.cuda.current_stream().cuda_stream)
    assert s == hom.HOM_OK, lib.hom_noalloc_last_error()
    torch.cuda.synchronize()
    assert torch.isfinite(out).all().item()


def test_noalloc_rejects_host_pointers_and_partial_overlap():
    from paper_1712_05145_gb300 import hom
    lib = hom.load_library()
    lib.hom_noalloc_last_error.restype = ctypes.c_char_p
    grid, nrhs = (32, 24, 16), 1
    ms, eps, E = _case(grid, nrhs)
    phase_dev = torch.from_numpy(ms.phase).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    host_out = torch.empty(eps.shape, dtype=torch.float64)
    s = _noalloc(lib, grid, phase_dev, ms.lame, ms.lam0, ms.mu0, nrhs, eps, E, host_out, stream)
    assert s == hom.HOM_ERR_ARG
    assert b"device" in lib.hom_noalloc_last_error()
    s = _noalloc(lib, grid, phase_dev, ms.lame, ms.lam0, ms.mu0, nrhs, eps.cpu(), E, torch.empty_like(eps), stream)
    assert s == hom.HOM_ERR_ARG
    big = torch.zeros((2,) + tuple(eps.shape[1:]), dtype=torch.float64, device="cuda")
    shifted = big.view(-1)[8:8 + eps.numel()].view(eps.shape)
    s = _noalloc(lib, grid, phase_dev, ms.lame, ms.lam0, ms.mu0, nrhs, big[:1], E, shifted, stream)
    assert s == hom.HOM_ERR_ARG
    assert b"overlap" in lib.hom_noalloc_last_error()


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1712_05145_gb300 import hom
    lib = hom.load_library()
    lib.hom_noalloc_last_error.restype = ctypes.c_char_p
    grid = (128, 64, 64)
    ms = synthetic.Microstructure(np.zeros((64, 64, 128), np.uint8), np.array([[1.0, 1.0]]), 1.0, 1.0)
    phase_dev = torch.from_numpy(ms.phase).cuda()
    eps = torch.zeros((1, 6, 64, 64, 128), dtype=torch.float64, device="cuda")
    out = torch.empty_like(eps)
    s = _noalloc(lib, grid, phase_dev, ms.lame, 1.0, 1.0, 1, eps, np.zeros((1, 6)), out,
                 torch.cuda.current_stream().cuda_stream)
    assert s == hom.HOM_ERR_SIZE
    assert b"scratch" in lib.hom_noalloc_last_error()
