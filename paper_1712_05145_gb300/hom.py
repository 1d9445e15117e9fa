"""Thin Python binding of libhom (include/hom.h): argument marshalling only.

Every computation runs in the CUDA library; this module only converts Python
arguments to pointers and sizes.  Device buffers are torch CUDA tensors (float64),
host buffers numpy arrays.  The functions keep the C names (``hom_create``,
``hom_solve``, ...); ``Homogenization`` wraps a handle for convenience.

Importing this module does not need a GPU; loading the library fails loudly if
``libhom.so`` has not been built (there is no CPU fallback).
"""
import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libhom.so")

HOM_OK = 0
HOM_ERR_ARG = 1
HOM_ERR_SIZE = 2
HOM_ERR_NOMEM = 3
HOM_ERR_NOT_CONVERGED = 4
HOM_ERR_ORDER = 5
HOM_ERR_NUMERIC = 6
HOM_ERR_TIMEOUT = 7
HOM_ERR_CUDA = 8

HOM_FP64 = 0
HOM_FP32_REFINE = 1
HOM_BASIC = 0
HOM_CG = 1
HOM_BICGSTAB = 2
HOM_POLARIZATION = 3
HOM_FIELD_STRAIN = 0
HOM_FIELD_DISPLACEMENT = 1
HOM_FIELD_STRESS = 2
HOM_GREEN_SPECTRAL = 0
HOM_GREEN_ROTATED = 1

HOM_KERNEL_PLANE_FWD = 0
HOM_KERNEL_ZPASS = 1
HOM_KERNEL_PLANE_INV = 2
HOM_KERNEL_COUNT = 8
KERNEL_NAMES = ["plane_fwd", "zpass", "plane_inv", "plane_fwd_f64", "zpass_f64", "plane_inv_f64",
                "ypass", "ypass_f64"]

EXPORTED = ["hom_default_options", "hom_create", "hom_solve", "hom_effective", "hom_get_field",
            "hom_ls_apply", "hom_equilibrium_error", "hom_fft_forward", "hom_fft_inverse", "hom_green_apply", "hom_profile",
            "hom_profile_read", "hom_ls_apply_noalloc", "hom_noalloc_last_error", "hom_estimate_bytes",
            "hom_server_create", "hom_server_create_batched", "hom_server_counters", "hom_server_submit", "hom_server_poll", "hom_server_wait", "hom_server_stats",
            "hom_server_destroy", "hom_device_bytes", "hom_launch_config", "hom_zpass_config", "hom_ypass_config", "hom_plane_config", "hom_set_rve",
            "hom_launch_count",
            "hom_last_error",
            "hom_status_string", "hom_destroy"]


class hom_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("scheme", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("max_refine", ctypes.c_int32), ("rhs_chunk", ctypes.c_int32),
                ("spectrum_budget_bytes", ctypes.c_int64), ("cuda_stream", ctypes.c_void_p),
                ("pass_mode", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("polarization_variant", ctypes.c_int32), ("z_mode", ctypes.c_int32),
                ("green_operator", ctypes.c_int32), ("n_rve", ctypes.c_int32), ("y_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 1)]


class hom_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("rel_residual_fp64", ctypes.c_double)]

    def as_dict(self):
        return {"iterations": self.iterations, "refinements": self.refinements, "status": self.status,
                "rel_residual": self.rel_residual, "rel_residual_fp64": self.rel_residual_fp64}


class hom_kernel_stat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("bytes", ctypes.c_int64), ("voxel_comps", ctypes.c_int64),
                ("ms", ctypes.c_double)]


class hom_request(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32 * 3), ("phase", ctypes.c_void_p), ("n_phase", ctypes.c_int32),
                ("lame", ctypes.c_void_p), ("lambda0", ctypes.c_double), ("mu0", ctypes.c_double),
                ("order", ctypes.c_int32), ("precision", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("tol", ctypes.c_double)]


class hom_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("order", ctypes.c_int32), ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("c_eff", ctypes.c_double * 36), ("d1", ctypes.c_double * 108),
                ("message", ctypes.c_char * 160)]

    def as_dict(self):
        return {"done": self.done, "status": self.status, "iterations": self.iterations, "order": self.order,
                "queue_ms": self.queue_ms, "run_ms": self.run_ms, "latency_ms": self.latency_ms,
                "c_eff": np.array(self.c_eff[:]).reshape(6, 6),
                "d1": np.array(self.d1[:]).reshape(6, 18) if self.order >= 1 else None,
                "message": self.message.decode(errors="replace")}


class HomError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (status_name(status), msg))
        self.status = status


_lib = None


def load_library(path=None):
    """Loads libhom.so (raises if it is missing: build it with paper_1712_05145_gb300.build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libhom.so not found at %s; run `python -m paper_1712_05145_gb300.build`" % p)
    lib = ctypes.CDLL(p)
    V, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.hom_default_options.argtypes = [ctypes.POINTER(hom_options)]
    lib.hom_default_options.restype = None
    lib.hom_create.argtypes = [ctypes.POINTER(ctypes.c_int32), V, I32, V, D, D, ctypes.POINTER(hom_options),
                               ctypes.POINTER(V)]
    lib.hom_create.restype = I32
    lib.hom_solve.argtypes = [V, I32, I32, V, D, V]
    lib.hom_solve.restype = I32
    lib.hom_effective.argtypes = [V, I32, V]
    lib.hom_effective.restype = I32
    lib.hom_get_field.argtypes = [V, I32, I32, I32, V, I32]
    lib.hom_get_field.restype = I32
    lib.hom_ls_apply.argtypes = [V, I32, V, V, V]
    lib.hom_ls_apply.restype = I32
    lib.hom_equilibrium_error.argtypes = [V, I32, V, V, V]
    lib.hom_equilibrium_error.restype = I32
    lib.hom_fft_forward.argtypes = [V, I32, V, V]
    lib.hom_fft_forward.restype = I32
    lib.hom_fft_inverse.argtypes = [V, I32, V, V]
    lib.hom_fft_inverse.restype = I32
    lib.hom_green_apply.argtypes = [V, I32, V, V]
    lib.hom_green_apply.restype = I32
    lib.hom_profile.argtypes = [V, I32]
    lib.hom_profile.restype = I32
    lib.hom_profile_read.argtypes = [V, V]
    lib.hom_profile_read.restype = I32
    lib.hom_ls_apply_noalloc.argtypes = [ctypes.POINTER(ctypes.c_int32), V, I32, V, D, D, I32, V, V, V, V]
    lib.hom_ls_apply_noalloc.restype = I32
    lib.hom_noalloc_last_error.argtypes = []
    lib.hom_noalloc_last_error.restype = ctypes.c_char_p
    lib.hom_estimate_bytes.argtypes = [ctypes.POINTER(ctypes.c_int32), I32, I32]
    lib.hom_estimate_bytes.restype = I64
    lib.hom_server_create.argtypes = [I64, I32, ctypes.POINTER(V)]
    lib.hom_server_create.restype = I32
    lib.hom_server_create_batched.argtypes = [I64, I32, I32, ctypes.POINTER(V)]
    lib.hom_server_create_batched.restype = I32
    lib.hom_server_counters.argtypes = [V, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.hom_server_counters.restype = I32
    lib.hom_server_submit.argtypes = [V, ctypes.POINTER(hom_request), ctypes.POINTER(I64)]
    lib.hom_server_submit.restype = I32
    lib.hom_server_poll.argtypes = [V, I64, ctypes.POINTER(hom_result)]
    lib.hom_server_poll.restype = I32
    lib.hom_server_wait.argtypes = [V, I64, ctypes.POINTER(hom_result)]
    lib.hom_server_wait.restype = I32
    lib.hom_server_stats.argtypes = [V, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.hom_server_stats.restype = I32
    lib.hom_server_destroy.argtypes = [V]
    lib.hom_server_destroy.restype = None
    lib.hom_device_bytes.argtypes = [V]
    lib.hom_device_bytes.restype = I64
    lib.hom_launch_config.argtypes = [V, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    lib.hom_launch_config.restype = ctypes.c_int
    lib.hom_set_rve.argtypes = [V, I32, V, I32, V, ctypes.c_double, ctypes.c_double]
    lib.hom_set_rve.restype = I32
    lib.hom_plane_config.argtypes = [V, ctypes.POINTER(ctypes.c_int32)]
    lib.hom_plane_config.restype = ctypes.c_int
    lib.hom_ypass_config.argtypes = [V, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    lib.hom_ypass_config.restype = ctypes.c_int
    lib.hom_zpass_config.argtypes = [V, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    lib.hom_zpass_config.restype = ctypes.c_int
    lib.hom_launch_count.argtypes = []
    lib.hom_launch_count.restype = I64
    lib.hom_last_error.argtypes = [V]
    lib.hom_last_error.restype = ctypes.c_char_p
    lib.hom_status_string.argtypes = [I32]
    lib.hom_status_string.restype = ctypes.c_char_p
    lib.hom_destroy.argtypes = [V]
    lib.hom_destroy.restype = None
    if path is None:
        _lib = lib
    return lib


def status_name(s):
    return load_library().hom_status_string(int(s)).decode()


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(x))


def _check(h, s):
    if s != HOM_OK:
        msg = load_library().hom_last_error(h).decode() if h else ""
        raise HomError(s, msg)


# ---- C-named functions ---------------------------------------------------------------
def hom_default_options():
    o = hom_options()
    load_library().hom_default_options(ctypes.byref(o))
    return o


def hom_create(grid, phase, lame, lambda0, mu0, options=None):
    """Returns a handle (ctypes c_void_p).  ``phase`` uint8 [N3][N2][N1] numpy or torch."""
    lib = load_library()
    g = (ctypes.c_int32 * 3)(*[int(v) for v in grid])
    lame = np.ascontiguousarray(lame, dtype=np.float64)
    if isinstance(phase, np.ndarray):
        phase = np.ascontiguousarray(phase, dtype=np.uint8)
    h = ctypes.c_void_p()
    opt = options if options is not None else hom_default_options()
    s = lib.hom_create(g, _ptr(phase), int(lame.shape[0]), _ptr(lame), float(lambda0), float(mu0),
                       ctypes.byref(opt), ctypes.byref(h))
    if s != HOM_OK:
        raise HomError(s, "hom_create rejected grid=%s" % (tuple(grid),))
    return h


def loads_of_order(order):
    """Unit loads of an order: 6 for order 0, 6 (o+1)(o+2)/2 for order o >= 1."""
    return 6 if order == 0 else 6 * (order + 1) * (order + 2) // 2


def hom_solve(h, order, tol, loads=None, n_loads=None):
    """Returns a list of per-load info dicts; raises HomError on any failure except
    non-convergence, which is reported through each load's status.  n_loads (with loads None)
    is the load count of a handle with several RVE slots: 6 x the slots to solve."""
    lib = load_library()
    nl = loads_of_order(order) if loads is None else int(np.asarray(loads).shape[0])
    if loads is None and n_loads is not None:
        nl = int(n_loads)
    arr = None
    if loads is not None:
        arr = np.ascontiguousarray(loads, dtype=np.float64).reshape(nl, 6 if order == 0 else 18)
    info = (hom_solve_info * nl)()
    s = lib.hom_solve(h, int(order), nl, _ptr(arr), float(tol), ctypes.cast(info, ctypes.c_void_p))
    if s not in (HOM_OK, HOM_ERR_NOT_CONVERGED):
        _check(h, s)
    return [i.as_dict() for i in info]


def hom_effective(h, order, nloads):
    out = np.zeros((6, nloads), dtype=np.float64)
    _check(h, load_library().hom_effective(h, int(order), _ptr(out)))
    return out


def hom_get_field(h, order, load, kind, dst, dst_on_device):
    _check(h, load_library().hom_get_field(h, int(order), int(load), int(kind), _ptr(dst), int(dst_on_device)))
    return dst


def hom_ls_apply(h, nrhs, eps_in, E, eps_out):
    E = None if E is None else np.ascontiguousarray(E, dtype=np.float64).reshape(nrhs, 6)
    _check(h, load_library().hom_ls_apply(h, int(nrhs), _ptr(eps_in), _ptr(E), _ptr(eps_out)))
    return eps_out


def hom_equilibrium_error(h, nrhs, eps=None, E=None):
    """Equilibrium error sqrt(<|div sigma|^2>) / |<sigma>| of sigma = C : (E + eps) per field, or
    of the solved order-0 loads when eps is None (nrhs = their count)."""
    E = None if (E is None or eps is None) else np.ascontiguousarray(E, dtype=np.float64).reshape(nrhs, 6)
    out = np.zeros(int(nrhs), dtype=np.float64)
    _check(h, load_library().hom_equilibrium_error(h, int(nrhs), _ptr(eps), _ptr(E), _ptr(out)))
    return out


def hom_fft_forward(h, nfield, f, fhat):
    _check(h, load_library().hom_fft_forward(h, int(nfield), _ptr(f), _ptr(fhat)))
    return fhat


def hom_fft_inverse(h, nfield, fhat, f):
    _check(h, load_library().hom_fft_inverse(h, int(nfield), _ptr(fhat), _ptr(f)))
    return f


def hom_green_apply(h, nrhs, tau_hat, eta_hat):
    _check(h, load_library().hom_green_apply(h, int(nrhs), _ptr(tau_hat), _ptr(eta_hat)))
    return eta_hat


def hom_profile(h, enable):
    _check(h, load_library().hom_profile(h, int(bool(enable))))


def hom_profile_read(h):
    """Per-kernel counters: list of dicts (launches, bytes, voxel_comps, ms) by kernel kind."""
    out = (hom_kernel_stat * HOM_KERNEL_COUNT)()
    _check(h, load_library().hom_profile_read(h, ctypes.cast(out, ctypes.c_void_p)))
    return [{"kernel": KERNEL_NAMES[k], "launches": out[k].launches, "bytes": out[k].bytes,
             "voxel_comps": out[k].voxel_comps, "ms": out[k].ms} for k in range(HOM_KERNEL_COUNT)]


def hom_ls_apply_noalloc(grid, phase_dev, lame, lambda0, mu0, nrhs, eps_in, E, eps_out, stream=None):
    """The allocation-free LS step (see include/hom.h); phase_dev, eps_in, eps_out on the device."""
    lib = load_library()
    g = (ctypes.c_int32 * 3)(*[int(v) for v in grid])
    lame = np.ascontiguousarray(lame, dtype=np.float64)
    E = None if E is None else np.ascontiguousarray(E, dtype=np.float64).reshape(nrhs, 6)
    s = lib.hom_ls_apply_noalloc(g, _ptr(phase_dev), int(lame.shape[0]), _ptr(lame), float(lambda0), float(mu0),
                                 int(nrhs), _ptr(eps_in), _ptr(E), _ptr(eps_out), stream)
    if s != HOM_OK:
        raise HomError(s, lib.hom_noalloc_last_error().decode())
    return eps_out


def hom_noalloc_last_error():
    return load_library().hom_noalloc_last_error().decode()


def hom_estimate_bytes(grid, order, precision=HOM_FP32_REFINE):
    g = (ctypes.c_int32 * 3)(*[int(v) for v in grid])
    return int(load_library().hom_estimate_bytes(g, int(order), int(precision)))


def hom_server_create(budget_bytes=0, max_active=4, max_batch=8):
    """A request server; max_batch order-0 requests of one grid share a handle and its launches."""
    s = ctypes.c_void_p()
    st = load_library().hom_server_create_batched(int(budget_bytes), int(max_active), int(max_batch),
                                                  ctypes.byref(s))
    if st != HOM_OK:
        raise HomError(st, "hom_server_create")
    return s


def hom_server_submit(s, ms, order=0, tol=1e-6, precision=HOM_FP32_REFINE, scheme=HOM_CG):
    """Queues the RVE ``ms`` (a synthetic.Microstructure); returns the request id."""
    n3, n2, n1 = ms.phase.shape
    phase = np.ascontiguousarray(ms.phase, dtype=np.uint8)
    lame = np.ascontiguousarray(ms.lame, dtype=np.float64)
    q = hom_request()
    q.grid[:] = [n1, n2, n3]
    q.phase = phase.ctypes.data
    q.n_phase = lame.shape[0]
    q.lame = lame.ctypes.data
    q.lambda0, q.mu0 = float(ms.lam0), float(ms.mu0)
    q.order, q.precision, q.scheme, q.tol = int(order), int(precision), int(scheme), float(tol)
    rid = ctypes.c_int64()
    st = load_library().hom_server_submit(s, ctypes.byref(q), ctypes.byref(rid))
    if st != HOM_OK:
        raise HomError(st, "hom_server_submit")
    return rid.value


def hom_server_poll(s, rid):
    r = hom_result()
    _check(None, load_library().hom_server_poll(s, int(rid), ctypes.byref(r)))
    return r.as_dict()


def hom_server_wait(s, rid):
    r = hom_result()
    _check(None, load_library().hom_server_wait(s, int(rid), ctypes.byref(r)))
    return r.as_dict()


def hom_server_stats(s):
    q, r, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(None, load_library().hom_server_stats(s, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)))
    return {"queued": q.value, "running": r.value, "bytes_in_use": b.value}


def hom_server_counters(s):
    """Batches run, requests run in them and handles created by a server so far."""
    b, r, h = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(None, load_library().hom_server_counters(s, ctypes.byref(b), ctypes.byref(r), ctypes.byref(h)))
    return {"batches": b.value, "requests": r.value, "handles_created": h.value}


def hom_server_destroy(s):
    if s:
        load_library().hom_server_destroy(s)


def hom_device_bytes(h):
    return int(load_library().hom_device_bytes(h))


def hom_launch_config(h):
    """(loads per launch, z-pass tile log2 width or -1) of a handle's iteration passes."""
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(h, load_library().hom_launch_config(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hom_set_rve(h, slot, phase, lame, lambda0, mu0):
    """Replaces RVE slot `slot` of a handle (phase uint8 [N3][N2][N1] numpy or torch, lame [n][2])."""
    lame = np.ascontiguousarray(lame, dtype=np.float64)
    if isinstance(phase, np.ndarray):
        phase = np.ascontiguousarray(phase, dtype=np.uint8)
    _check(h, load_library().hom_set_rve(h, int(slot), _ptr(phase), int(lame.shape[0]), _ptr(lame),
                                         float(lambda0), float(mu0)))


def hom_plane_config(h):
    """CTAs per plane of the cluster plane passes of a handle's FP32 transforms (0: not used)."""
    a = ctypes.c_int32()
    _check(h, load_library().hom_plane_config(h, ctypes.byref(a)))
    return a.value


def hom_ypass_config(h):
    """(tile log2 width or -1, 1 if its FP32 tiles move by TMA else 0) of a handle's split y pass."""
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(h, load_library().hom_ypass_config(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hom_zpass_config(h):
    """(z stage, tile log2 width or -1) of a handle's iteration passes; the z stage is 1 for the
    cluster z pass, 2 for its TMA form, 0 for the single-CTA z pass."""
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(h, load_library().hom_zpass_config(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hom_launch_count():
    """Kernels the library has launched in this process (host-side count)."""
    return int(load_library().hom_launch_count())


def hom_last_error(h):
    return load_library().hom_last_error(h).decode()


def hom_destroy(h):
    if h:
        load_library().hom_destroy(h)


# ---- convenience wrapper ---------------------------------------------------------------
class Homogenization:
    """One RVE on the GPU.  ``ms`` is a synthetic.Microstructure (or anything with
    .phase, .lame, .lam0, .mu0)."""


    def __init__(self, ms, precision=HOM_FP32_REFINE, scheme=HOM_CG, max_iter=2000, check_every=8,
                 max_refine=6, rhs_chunk=0, spectrum_budget_bytes=1024 << 20, stream=None, lam0=None, mu0=None,
                 pass_mode=0, autotune=0, polarization_variant=0, z_mode=0, green_operator=0, n_rve=1,
                 y_mode=0):
        n3, n2, n1 = ms.phase.shape
        self.grid = (n1, n2, n3)
        self.M = n1 * n2 * n3
        opt = hom_default_options()
        opt.precision = precision
        opt.scheme = scheme
        opt.max_iter = max_iter
        opt.check_every = check_every
        opt.max_refine = max_refine
        opt.rhs_chunk = rhs_chunk
        opt.spectrum_budget_bytes = spectrum_budget_bytes
        opt.cuda_stream = stream
        opt.pass_mode = pass_mode
        opt.autotune = autotune
        opt.polarization_variant = polarization_variant
        opt.z_mode = z_mode
        opt.green_operator = green_operator
        opt.n_rve = n_rve
        opt.y_mode = y_mode
        self.h = hom_create(self.grid, ms.phase, ms.lame, ms.lam0 if lam0 is None else lam0,
                            ms.mu0 if mu0 is None else mu0, opt)
        self.nloads = {}

    def close(self):
        if self.h:
            hom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, order, tol, loads=None, n_loads=None):
        info = hom_solve(self.h, order, tol, loads, n_loads)
        self.nloads[order] = len(info)
        return info

    def effective(self, order):
        return hom_effective(self.h, order, self.nloads[order])

    def equilibrium_error(self):
        """Equilibrium error of the solved order-0 loads (one value per load)."""
        return hom_equilibrium_error(self.h, self.nloads.get(0, 0))

    def field(self, order, load, kind=HOM_FIELD_STRAIN, device=False):
        nc = 3 if kind == HOM_FIELD_DISPLACEMENT else 6
        n1, n2, n3 = self.grid
        if device:
            import torch
            dst = torch.empty((nc, n3, n2, n1), dtype=torch.float64, device="cuda")
            return hom_get_field(self.h, order, load, kind, dst, 1)
        dst = np.empty((nc, n3, n2, n1), dtype=np.float64)
        return hom_get_field(self.h, order, load, kind, dst, 0)
