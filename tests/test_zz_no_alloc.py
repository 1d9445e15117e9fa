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


def _noalloc(lib, grid, phase_dev, lame, lam0, mu0, nrhs, eps_in, E, out, stream):
    g = (ctypes.c_int32 * 3)(*grid)
    lame = np.ascontiguousarray(lame, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    fn = lib.hom_ls_apply_noalloc
    fn.restype = ctypes.c_int32
    fn.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                   ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn(g, ctypes.c_void_p(phase_dev.data_ptr()), lame.shape[0], ctypes.c_void_p(lame.ctypes.data),
              lam0, mu0, nrhs, ctypes.c_void_p(eps_in.data_ptr()), ctypes.c_void_p(E.ctypes.data),
              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_step_matches_ls_apply_on_two_calls():
    from paper_1712_05145_gb300 import hom
    lib = hom.load_library()
    grid = (32, 24, 16)
    n1, n2, n3 = grid
    ms = synthetic.Microstructure(random_phase(grid, 3, 31), np.array([[1.0, 1.0], [8.0, 5.0], [0.4, 0.3]]),
                                  3.0, 2.0)
    nrhs = 3
    eps = torch.from_numpy(random_mandel_fields(nrhs, grid, 17)).cuda()
    E = np.random.default_rng(4).uniform(-1, 1, size=(nrhs, 6))
    H = hom.Homogenization(ms, precision=hom.HOM_FP64)
    ref = torch.empty_like(eps)
    hom.hom_ls_apply(H.h, nrhs, eps, E, ref)
    H.close()
    phase_dev = torch.from_numpy(ms.phase).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full_like(eps, float("nan"))
        s = _noalloc(lib, grid, phase_dev, ms.lame, ms.lam0, ms.mu0, nrhs, eps, E, out, stream)
        assert s == hom.HOM_OK, lib.hom_noalloc_last_error()
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-12, err


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
