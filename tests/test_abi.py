"""The C-ABI library loads and exports every entry point its header declares (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1712_05145_gb300 import build, hom

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return hom.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hom.h")).read()
    return sorted(set(re.findall(r"HOM_API\s+[\w\s\*]+?\b(hom_\w+)\s*\(", text)))


def test_header_declares_the_bound_functions():
    assert declared_symbols() == sorted(hom.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings_and_defaults(lib):
    assert hom.status_name(hom.HOM_ERR_SIZE) == "HOM_ERR_SIZE"
    o = hom.hom_default_options()
    assert o.precision == hom.HOM_FP32_REFINE and o.scheme == hom.HOM_CG and o.check_every == 8


@pytest.mark.parametrize("grid", [(7, 8, 8), (10, 8, 8), (8, 5, 8), (8, 8, 10), (2, 8, 8), (2048, 32, 32)])
def test_unsupported_grids_rejected_before_any_cuda_call(lib, grid):
    n1, n2, n3 = grid
    phase = np.zeros((n3, n2, n1), dtype=np.uint8)
    with pytest.raises(hom.HomError) as e:
        hom.hom_create(grid, phase, np.array([[1.0, 1.0]]), 1.0, 1.0)
    assert e.value.status == hom.HOM_ERR_SIZE


def test_fused_only_mode_rejects_planes_larger_than_one_cta(lib):
    phase = np.zeros((8, 128, 256), dtype=np.uint8)
    opt = hom.hom_default_options()
    opt.pass_mode = 1
    with pytest.raises(hom.HomError) as e:
        hom.hom_create((256, 128, 8), phase, np.array([[1.0, 1.0]]), 1.0, 1.0, opt)
    assert e.value.status == hom.HOM_ERR_SIZE
    opt.pass_mode = 4
    with pytest.raises(hom.HomError) as e:
        hom.hom_create((8, 8, 8), np.zeros((8, 8, 8), np.uint8), np.array([[1.0, 1.0]]), 1.0, 1.0, opt)
    assert e.value.status == hom.HOM_ERR_ARG
    opt.pass_mode = 0
    opt.z_mode = 4
    with pytest.raises(hom.HomError) as e:
        hom.hom_create((8, 8, 8), np.zeros((8, 8, 8), np.uint8), np.array([[1.0, 1.0]]), 1.0, 1.0, opt)
    assert e.value.status == hom.HOM_ERR_ARG
    opt.z_mode = 0
    opt.y_mode = 3
    with pytest.raises(hom.HomError) as e:
        hom.hom_create((8, 8, 8), np.zeros((8, 8, 8), np.uint8), np.array([[1.0, 1.0]]), 1.0, 1.0, opt)
    assert e.value.status == hom.HOM_ERR_ARG


def test_bad_reference_medium_rejected(lib):
    phase = np.zeros((8, 8, 8), dtype=np.uint8)
    for lam0, mu0 in [(1.0, 0.0), (-2.0, 1.0)]:
        with pytest.raises(hom.HomError) as e:
            hom.hom_create((8, 8, 8), phase, np.array([[1.0, 1.0]]), lam0, mu0)
        assert e.value.status == hom.HOM_ERR_ARG


def test_polarization_scheme_rejects_expanding_arguments(lib):
    """The polarization scheme contracts only for positive reference moduli and non-negative
    phase moduli; anything else, and an unknown variant, is refused before any CUDA call."""
    phase = np.zeros((8, 8, 8), dtype=np.uint8)
    cases = [((1.0, 1.0), 1.0, -0.5, 0),     # mu0 < 0
             ((1.0, 1.0), -1.0, 0.4, 0),     # 3 lam0 + 2 mu0 < 0
             ((-1.0, 0.2), 1.0, 1.0, 0),     # a phase with 3K < 0
             ((1.0, 1.0), 1.0, 1.0, 2)]      # unknown variant
    for (lam, mu), lam0, mu0, variant in cases:
        opt = hom.hom_default_options()
        opt.scheme = hom.HOM_POLARIZATION
        opt.polarization_variant = variant
        with pytest.raises(hom.HomError) as e:
            hom.hom_create((8, 8, 8), phase, np.array([[lam, mu]]), lam0, mu0, opt)
        assert e.value.status == hom.HOM_ERR_ARG


def test_null_handle_calls(lib):
    assert lib.hom_solve(None, 0, 6, None, 1e-6, None) == hom.HOM_ERR_ARG
    assert lib.hom_effective(None, 0, None) == hom.HOM_ERR_ARG
    assert lib.hom_device_bytes(None) == 0
    lib.hom_destroy(None)


def test_estimate_accepts_two_dimensional_cells_and_rejects_empty_axes(lib):
    assert hom.hom_estimate_bytes((64, 64, 1), 0) > 0
    for o in range(1, 7):
        assert hom.hom_estimate_bytes((64, 64, 1), o) > hom.hom_estimate_bytes((64, 64, 1), o - 1)
    for g in [(0, 8, 8), (8, 0, 8), (8, 8, 0), (8, 1, 8), (1, 8, 8)]:
        assert hom.hom_estimate_bytes(g, 0) < 0
    assert hom.hom_estimate_bytes((8, 8, 8), 7) < 0
    assert hom.hom_estimate_bytes((8, 8, 8), -1) < 0
