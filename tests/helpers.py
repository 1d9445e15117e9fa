"""Shared helpers of the GPU parity tests: seeded inputs and oracle-side conversions."""
import numpy as np

from oracle.tensors import mandel_to_tensor, tensor_to_mandel

# FP64 and FP32 parity tolerances (max-norm error relative to the max-norm of the oracle)
TOL = {0: 1e-10, 1: 1e-5}          # keyed by hom precision: 0 = FP64, 1 = FP32 + refinement
TOL_FFT = {0: 1e-12, 1: 2e-6}
TOL_EFF = {0: 1e-9, 1: 1e-6}


def rel_err(got, ref):
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def random_mandel_fields(n, grid, seed):
    n1, n2, n3 = grid
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, size=(n, 6, n3, n2, n1))


def oracle_ls_step_mandel(pb, eps_m, E_m):
    """Oracle LS step on Mandel inputs (one load)."""
    return tensor_to_mandel(pb.ls_step(mandel_to_tensor(eps_m), mandel_to_tensor(E_m)))


def random_phase(grid, nphase, seed, p=None):
    n1, n2, n3 = grid
    rng = np.random.default_rng(seed)
    return rng.choice(nphase, size=(n3, n2, n1), p=p).astype(np.uint8)
