"""ctypes binding of libstglbm.so, one Python function per C entry point.

Argument marshalling only: every step of the computation runs in the CUDA
library.  There is no fallback; if the shared library is missing or cannot be
loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstglbm.so")

STG_OK, STG_ERR_INVALID, STG_ERR_NOMEM, STG_ERR_UNSTABLE, STG_ERR_TIMEOUT, STG_ERR_CUDA = range(6)
STG_FP32, STG_FP16_SHIFTED, STG_FP16_SHIFTED_SR = 0, 1, 2
STG_REGULARIZED, STG_BGK = 0, 1
STG_BC_X_INLET_OUTLET, STG_BC_X_PERIODIC = 0, 1
STG_BC_Y_WALLS, STG_BC_Y_PERIODIC = 0, 1
STG_STREAM_PULL, STG_STREAM_AA = 0, 1

c_double_p = C.POINTER(C.c_double)


class stg_domain(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("storage", C.c_int32),
                ("collision", C.c_int32), ("bc_x", C.c_int32), ("bc_y", C.c_int32),
                ("stats_every", C.c_int32), ("check_every", C.c_int32), ("streaming", C.c_int32),
                ("tau0", C.c_double), ("c_smag", C.c_double), ("force", C.c_double * 3),
                ("mass_tol", C.c_double), ("sponge_len", C.c_double), ("sponge_K", C.c_double),
                ("sponge_p", C.c_double)]


class stg_rans_profile(C.Structure):
    _fields_ = [("n_fv", C.c_int32), ("pad0", C.c_int32), ("y_c", c_double_p), ("U", c_double_p),
                ("k", c_double_p), ("eps", c_double_p), ("R", c_double_p), ("U_bulk", C.c_double),
                ("nu_phys", C.c_double), ("h_phys", C.c_double), ("mach_target", C.c_double)]


class stg_params(C.Structure):
    _fields_ = [("n_modes", C.c_int32), ("pad0", C.c_int32), ("C_l", C.c_double), ("alpha", C.c_double),
                ("T_filter", C.c_double)]


class stg_tile(C.Structure):
    _fields_ = [("interior_layout", C.c_int32), ("interior_zc", C.c_int32), ("wall_zc", C.c_int32),
                ("pad0", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class stg_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class stg_stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("n_samples", C.c_int64), ("mass", C.c_double), ("mass0", C.c_double),
                ("mean_sum", c_double_p), ("rey_sum", c_double_p)]


class stg_info(C.Structure):
    _fields_ = [("c_x", C.c_double), ("c_t", C.c_double), ("U_b", C.c_double), ("max_le", C.c_double),
                ("k_min", C.c_double), ("k_max", C.c_double), ("a_filter", C.c_double),
                ("n_modes", C.c_int64), ("device_bytes", C.c_int64)]


class stg_job(C.Structure):
    _fields_ = [("arrival_s", C.c_double), ("domain", C.POINTER(stg_domain)), ("rans", C.POINTER(stg_rans_profile)),
                ("stg", C.POINTER(stg_params)), ("seed", C.c_uint64), ("steps", C.c_int64),
                ("mean_sum", c_double_p), ("rey_sum", c_double_p)]


class stg_job_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("pad0", C.c_int32), ("admit_s", C.c_double), ("finish_s", C.c_double),
                ("latency_s", C.c_double), ("n_samples", C.c_int64), ("device_bytes", C.c_int64),
                ("mass", C.c_double), ("mass0", C.c_double)]


class stg_serve_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("max_active", C.c_int32), ("pad0", C.c_int32)]


class stg_serve_report(C.Structure):
    _fields_ = [("wall_s", C.c_double), ("jobs_per_s", C.c_double), ("aggregate_mlups", C.c_double),
                ("p50_latency_s", C.c_double), ("p99_latency_s", C.c_double), ("mean_latency_s", C.c_double),
                ("completed", C.c_int64), ("failed", C.c_int64), ("cell_updates", C.c_int64),
                ("peak_device_bytes", C.c_int64), ("peak_active", C.c_int32), ("pad0", C.c_int32)]


_SIGNATURES = {
    "stg_lbm_create": (C.c_int, [C.POINTER(stg_domain), C.POINTER(stg_rans_profile), C.POINTER(stg_params),
                                 C.c_uint64, C.POINTER(stg_allocator), C.c_void_p, C.POINTER(C.c_void_p)]),
    "stg_lbm_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "stg_lbm_step_timed": (C.c_int, [C.c_void_p, C.c_int64, c_double_p, c_double_p]),
    "stg_lbm_stats": (C.c_int, [C.c_void_p, C.POINTER(stg_stats)]),
    "stg_lbm_reset_stats": (C.c_int, [C.c_void_p]),
    "stg_lbm_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "stg_lbm_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int64]),
    "stg_lbm_get_inlet": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "stg_lbm_device_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "stg_lbm_info": (C.c_int, [C.c_void_p, C.POINTER(stg_info)]),
    "stg_lbm_set_tile": (C.c_int, [C.c_void_p, C.POINTER(stg_tile)]),
    "stg_lbm_get_tile": (C.c_int, [C.c_void_p, C.POINTER(stg_tile)]),
    "stg_lbm_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(stg_tile)]),
    "stg_lbm_checkpoint_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "stg_lbm_save": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "stg_lbm_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "stg_lbm_get_block": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                    C.c_void_p]),
    "stg_lbm_set_probes": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "stg_lbm_step_probed": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_float)]),
    "stg_lbm_estimate_bytes": (C.c_int, [C.POINTER(stg_domain), C.POINTER(stg_params), C.POINTER(C.c_int64)]),
    "stg_batch_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "stg_batch_add": (C.c_int, [C.c_void_p, C.c_void_p]),
    "stg_batch_remove": (C.c_int, [C.c_void_p, C.c_void_p]),
    "stg_batch_size": (C.c_int, [C.c_void_p]),
    "stg_batch_block_steps": (C.c_int, [C.c_void_p]),
    "stg_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "stg_batch_sync": (C.c_int, [C.c_void_p]),
    "stg_batch_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(stg_tile)]),
    "stg_batch_destroy": (None, [C.c_void_p]),
    "stg_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "stg_serve_run": (C.c_int, [C.POINTER(stg_job), C.c_int32, C.POINTER(stg_serve_config), C.c_void_p,
                                C.POINTER(stg_job_result), C.POINTER(stg_serve_report)]),
    "stg_serve_last_error": (C.c_char_p, []),
    "stg_lbm_destroy": (None, [C.c_void_p]),
    "stg_lbm_last_error": (C.c_char_p, [C.c_void_p]),
    "stg_mode_draws": (C.c_int, [C.c_uint64, C.c_int32, c_double_p]),
    "stg_lbm_version": (C.c_char_p, []),
    "stg_lattice_mass_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                           C.c_void_p]),
}

_lib = None


def lib():
    """Load libstglbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libstglbm.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class StgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _check(rc, handle=None):
    if rc != STG_OK:
        msg = lib().stg_lbm_last_error(handle)
        raise StgError(rc, msg.decode() if msg else "")
    return rc


# ---------------------------------------------------------------- raw entry points
def stg_lbm_create(domain, rans, params, seed, allocator=None, stream=0):
    h = C.c_void_p()
    rc = lib().stg_lbm_create(C.byref(domain), C.byref(rans) if rans is not None else None,
                              C.byref(params) if params is not None else None, seed,
                              C.byref(allocator) if allocator is not None else None, C.c_void_p(stream),
                              C.byref(h))
    _check(rc, None)
    return h


def stg_lbm_step(h, n):
    return _check(lib().stg_lbm_step(h, n), h)


def stg_lbm_step_timed(h, n):
    a = C.c_double()
    b = C.c_double()
    _check(lib().stg_lbm_step_timed(h, n, C.byref(a), C.byref(b)), h)
    return a.value, b.value


def stg_lbm_stats(h, mean_sum=None, rey_sum=None):
    s = stg_stats()
    s.mean_sum = mean_sum.ctypes.data_as(c_double_p) if mean_sum is not None else None
    s.rey_sum = rey_sum.ctypes.data_as(c_double_p) if rey_sum is not None else None
    rc = lib().stg_lbm_stats(h, C.byref(s))
    return rc, s


def stg_lbm_reset_stats(h):
    return _check(lib().stg_lbm_reset_stats(h), h)


def stg_lbm_get_state(h, out):
    return _check(lib().stg_lbm_get_state(h, C.c_void_p(out.ctypes.data), out.nbytes), h)


def stg_lbm_set_state(h, arr, step=0):
    return _check(lib().stg_lbm_set_state(h, C.c_void_p(arr.ctypes.data), arr.nbytes, step), h)


def stg_lbm_get_inlet(h, out):
    return _check(lib().stg_lbm_get_inlet(h, out.ctypes.data_as(C.POINTER(C.c_float))), h)


def stg_lbm_device_state(h):
    p = C.c_void_p()
    u = C.c_void_p()
    _check(lib().stg_lbm_device_state(h, C.byref(p), C.byref(u)), h)
    return p.value, u.value


def stg_lbm_info(h):
    i = stg_info()
    _check(lib().stg_lbm_info(h, C.byref(i)), h)
    return i


def stg_lbm_set_tile(h, layout, zc, wall_zc):
    t = stg_tile(layout, zc, wall_zc, 0)
    return _check(lib().stg_lbm_set_tile(h, C.byref(t)), h)


def stg_lbm_get_tile(h):
    t = stg_tile()
    _check(lib().stg_lbm_get_tile(h, C.byref(t)), h)
    return t.interior_layout, t.interior_zc, t.wall_zc


def stg_lbm_autotune(h, trial_passes=10):
    t = stg_tile()
    _check(lib().stg_lbm_autotune(h, trial_passes, C.byref(t)), h)
    return t.interior_layout, t.interior_zc, t.wall_zc


def stg_lbm_destroy(h):
    lib().stg_lbm_destroy(h)


def stg_lbm_last_error(h=None):
    m = lib().stg_lbm_last_error(h)
    return m.decode() if m else ""


def stg_mode_draws(seed, n):
    out = np.zeros(4 * n)
    _check(lib().stg_mode_draws(seed, n, out.ctypes.data_as(c_double_p)))
    return out


def stg_lbm_version():
    return lib().stg_lbm_version().decode()


def stg_lattice_mass_noalloc(pops_dev, storage, nx, ny, nz, mass_out_dev, stream=0):
    """Enqueue the FP64 mass of a device population field into mass_out_dev
    (a device double) without any allocation; returns the status code."""
    return lib().stg_lattice_mass_noalloc(C.c_void_p(pops_dev), storage, nx, ny, nz, C.c_void_p(mass_out_dev),
                                          C.c_void_p(stream))


# ---------------------------------------------------------------- estimate, batch, serving
def stg_lbm_estimate_bytes(domain, params=None):
    out = C.c_int64()
    _check(lib().stg_lbm_estimate_bytes(C.byref(domain), C.byref(params) if params is not None else None,
                                        C.byref(out)))
    return out.value


def _bcheck(rc, b):
    if rc != STG_OK:
        msg = lib().stg_batch_last_error(b)
        raise StgError(rc, msg.decode() if msg else "")
    return rc


def stg_batch_create(stream=0):
    b = C.c_void_p()
    _bcheck(lib().stg_batch_create(C.c_void_p(stream), C.byref(b)), None)
    return b


def stg_batch_add(b, h):
    return _bcheck(lib().stg_batch_add(b, h), b)


def stg_batch_remove(b, h):
    return _bcheck(lib().stg_batch_remove(b, h), b)


def stg_batch_size(b):
    return lib().stg_batch_size(b)


def stg_batch_block_steps(b):
    return lib().stg_batch_block_steps(b)


def stg_batch_step(b, n):
    return _bcheck(lib().stg_batch_step(b, n), b)


def stg_batch_sync(b):
    return _bcheck(lib().stg_batch_sync(b), b)


def stg_batch_autotune(b, trial_passes=10):
    t = stg_tile()
    _bcheck(lib().stg_batch_autotune(b, trial_passes, C.byref(t)), b)
    return t.interior_layout, t.interior_zc, t.wall_zc


def stg_batch_destroy(b):
    lib().stg_batch_destroy(b)


def stg_serve_run(jobs, cfg, stream=0):
    """jobs: a ctypes array of stg_job; returns (rc, results array, report)."""
    n = len(jobs)
    res = (stg_job_result * max(n, 1))()
    rep = stg_serve_report()
    rc = lib().stg_serve_run(jobs, n, C.byref(cfg), C.c_void_p(stream), res, C.byref(rep))
    if rc != STG_OK:
        msg = lib().stg_serve_last_error()
        raise StgError(rc, msg.decode() if msg else "")
    return res, rep


def stg_lbm_set_probes(h, xyz):
    a = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    return _check(lib().stg_lbm_set_probes(h, a.shape[0], a.ctypes.data_as(C.POINTER(C.c_int32))), h)


def stg_lbm_step_probed(h, n, n_probes):
    out = np.empty((n, n_probes, 3), dtype=np.float32)
    _check(lib().stg_lbm_step_probed(h, n, out.ctypes.data_as(C.POINTER(C.c_float))), h)
    return out


def stg_lbm_get_block(h, x0, y0, z0, out):
    """out: host array [19][bz][by][bx] of the storage dtype."""
    _, bz, by, bx = out.shape
    return _check(lib().stg_lbm_get_block(h, x0, y0, z0, bx, by, bz, C.c_void_p(out.ctypes.data)), h)


def stg_lbm_save(h):
    n = C.c_size_t()
    _check(lib().stg_lbm_checkpoint_bytes(h, C.byref(n)), h)
    out = np.empty(n.value, dtype=np.uint8)
    _check(lib().stg_lbm_save(h, C.c_void_p(out.ctypes.data), out.nbytes), h)
    return out


def stg_lbm_load(h, image):
    image = np.ascontiguousarray(image, dtype=np.uint8)
    return _check(lib().stg_lbm_load(h, C.c_void_p(image.ctypes.data), image.nbytes), h)
