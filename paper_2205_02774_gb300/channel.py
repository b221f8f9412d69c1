"""Channel: a Python handle over one libstglbm lattice.

PyTorch supplies the device memory (its caching allocator, through the C
allocator callbacks) and the CUDA stream; the computation itself runs in the
library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi as A

# D3Q19 weights of the documented population order (rest, axis, edge)
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


class _TorchAllocator:
    """stg_allocator backed by torch.cuda.caching_allocator_alloc/delete."""

    def __init__(self, torch, device, stream):
        self.torch = torch
        self.device = device
        self.stream = stream
        self._alloc = A.ALLOC_FN(self._do_alloc)
        self._free = A.FREE_FN(self._do_free)
        self.struct = A.stg_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, ctx):
        try:
            return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
        except Exception:  # allocation failure is reported to the library as NULL
            return None

    def _do_free(self, ptr, nbytes, ctx):
        self.torch.cuda.caching_allocator_delete(int(ptr))


def _domain(nx, ny, nz, storage, collision, bc_x, bc_y, stats_every, check_every, tau0, c_smag, force,
            mass_tol, sponge=(0.0, 1000.0, 3.0), streaming="pull"):
    d = A.stg_domain()
    d.streaming = {"pull": A.STG_STREAM_PULL, "aa": A.STG_STREAM_AA}[streaming]
    d.sponge_len, d.sponge_K, d.sponge_p = sponge
    d.nx, d.ny, d.nz = nx, ny, nz
    d.storage = {"fp32": A.STG_FP32, "fp16s": A.STG_FP16_SHIFTED, "fp16sr": A.STG_FP16_SHIFTED_SR}[storage]
    d.collision = {"regularized": A.STG_REGULARIZED, "bgk": A.STG_BGK}[collision]
    d.bc_x = {"stg": A.STG_BC_X_INLET_OUTLET, "periodic": A.STG_BC_X_PERIODIC}[bc_x]
    d.bc_y = {"walls": A.STG_BC_Y_WALLS, "periodic": A.STG_BC_Y_PERIODIC}[bc_y]
    d.stats_every, d.check_every = stats_every, check_every
    d.tau0, d.c_smag = tau0, c_smag
    d.force = (C.c_double * 3)(*force)
    d.mass_tol = mass_tol
    return d


def create_structs(nx, ny, nz, *, profile=None, tau0=0.52, c_smag=0.01, force=(0.0, 0.0, 0.0), storage="fp32",
                   collision="regularized", bc_x="stg", bc_y="walls", stats_every=0, check_every=0, mass_tol=0.0,
                   n_modes=100, C_l=3.0, alpha=0.01, t_filter=0.0, mach_target=0.0516, sponge=(0.0, 1000.0, 3.0),
                   streaming="pull"):
    """The stg_domain, stg_rans_profile and stg_params of a lattice (the last
    two None for periodic x), plus the arrays they point into (keep them
    alive while the structs are in use).  sponge = (length, K, p);
    streaming: "pull" (two lattices) or "aa" (one lattice in place)."""
    domain = _domain(nx, ny, nz, storage, collision, bc_x, bc_y, stats_every, check_every, tau0, c_smag, force,
                     mass_tol, sponge, streaming)
    keep = []
    rans = None
    params = None
    if bc_x == "stg":
        arrays = [np.ascontiguousarray(getattr(profile, k), dtype=np.float64) for k in ("y_c", "U", "k", "eps")]
        arrays.append(np.ascontiguousarray(profile.R, dtype=np.float64).reshape(-1))
        keep += arrays
        rans = A.stg_rans_profile()
        rans.n_fv = arrays[0].size
        rans.y_c, rans.U, rans.k, rans.eps, rans.R = [a.ctypes.data_as(A.c_double_p) for a in arrays]
        rans.U_bulk, rans.nu_phys, rans.h_phys = profile.U_bulk, profile.nu_phys, profile.h_phys
        rans.mach_target = mach_target
        params = A.stg_params()
        params.n_modes, params.C_l, params.alpha, params.T_filter = n_modes, C_l, alpha, t_filter
    return domain, rans, params, keep


def case_kwargs(case):
    """create_structs / Channel keyword arguments of a workload case."""
    return dict(profile=case.profile() if case.bc_x == "stg" else None, tau0=case.tau0, c_smag=case.c_smag,
                force=case.force, storage=case.storage, collision=case.collision, bc_x=case.bc_x, bc_y=case.bc_y,
                stats_every=case.stats_every, n_modes=case.n_modes, t_filter=case.t_filter,
                mach_target=case.mach_target, sponge=(case.sponge_len, case.sponge_K, case.sponge_p),
                streaming=case.streaming)


class Channel:
    """One STG-LBM lattice on the current CUDA device.

    ``profile`` needs attributes y_c, U, k, eps, R (n x 6), U_bulk, nu_phys,
    h_phys (a RANS interface profile in physical units)."""

    def __init__(self, nx, ny, nz, *, profile=None, tau0=0.52, c_smag=0.01, force=(0.0, 0.0, 0.0),
                 storage="fp32", collision="regularized", bc_x="stg", bc_y="walls", stats_every=0,
                 check_every=0, mass_tol=0.0, n_modes=100, C_l=3.0, alpha=0.01, t_filter=0.0,
                 mach_target=0.0516, seed=0, stream=None, use_torch_allocator=True, sponge=(0.0, 1000.0, 3.0),
                 streaming="pull"):
        import torch
        self.torch = torch
        self.nx, self.ny, self.nz = nx, ny, nz
        self.storage = storage
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.domain, rans, params, self._keep = create_structs(
            nx, ny, nz, profile=profile, tau0=tau0, c_smag=c_smag, force=force, storage=storage,
            collision=collision, bc_x=bc_x, bc_y=bc_y, stats_every=stats_every, check_every=check_every,
            mass_tol=mass_tol, n_modes=n_modes, C_l=C_l, alpha=alpha, t_filter=t_filter, mach_target=mach_target,
            sponge=sponge, streaming=streaming)
        self._allocator = _TorchAllocator(torch, self.device, self.stream) if use_torch_allocator else None
        self.h = A.stg_lbm_create(self.domain, rans, params, seed,
                                  self._allocator.struct if self._allocator else None, self.stream.cuda_stream)

    @classmethod
    def from_case(cls, case, **kw):
        args = case_kwargs(case)
        args["seed"] = case.seed
        args.update(kw)
        return cls(case.nx, case.ny, case.nz, **args)

    # ------------------------------------------------------------------
    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    @property
    def state_dtype(self):
        return np.float32 if self.storage == "fp32" else np.uint16

    @property
    def shape(self):
        return (19, self.nz, self.ny, self.nx)

    def step(self, n=1):
        A.stg_lbm_step(self.h, n)

    def set_tile(self, layout, zc, wall_zc):
        A.stg_lbm_set_tile(self.h, layout, zc, wall_zc)

    def tile(self):
        return A.stg_lbm_get_tile(self.h)

    def autotune(self, trial_passes=10):
        return A.stg_lbm_autotune(self.h, trial_passes)

    def set_probes(self, xyz):
        self._n_probes = int(np.asarray(xyz).reshape(-1, 3).shape[0])
        A.stg_lbm_set_probes(self.h, xyz)

    def step_probed(self, n):
        """n steps; returns the probe velocities after each, shape (n, n_probes, 3)."""
        return A.stg_lbm_step_probed(self.h, n, self._n_probes)

    def step_timed(self, n):
        return A.stg_lbm_step_timed(self.h, n)

    def get_state(self):
        out = np.empty(self.shape, dtype=self.state_dtype)
        A.stg_lbm_get_state(self.h, out)
        return out

    def save(self):
        """Checkpoint image (numpy uint8) of the whole evolving state."""
        return A.stg_lbm_save(self.h)

    def load(self, image):
        A.stg_lbm_load(self.h, image)

    def get_block(self, x0, y0, z0, bx, by, bz):
        """Sub-block [19][bz][by][bx] of the current populations (storage format)."""
        out = np.empty((19, bz, by, bx), dtype=self.state_dtype)
        A.stg_lbm_get_block(self.h, x0, y0, z0, out)
        return out

    def set_state(self, arr, step=0):
        arr = np.ascontiguousarray(arr, dtype=self.state_dtype)
        assert arr.shape == self.shape
        A.stg_lbm_set_state(self.h, arr, step)

    def encode(self, f):
        """Storage format (g_i = f_i - w_i as float32 or binary16 bits) of populations f."""
        g = np.asarray(f, dtype=np.float64) - W19[:, None, None, None]
        if self.storage == "fp32":
            return np.ascontiguousarray(g.astype(np.float32))
        return np.ascontiguousarray(g.astype(np.float16).view(np.uint16))

    def decode(self, s):
        """float64 populations f_i from the storage format."""
        g = s.astype(np.float64) if self.storage == "fp32" else s.view(np.float16).astype(np.float64)
        return g + W19[:, None, None, None]

    def populations(self):
        """Current populations as float64 f_i (decoded from the storage format)."""
        return self.decode(self.get_state())

    def inlet(self):
        out = np.empty((3, self.nz, self.ny), dtype=np.float32)
        A.stg_lbm_get_inlet(self.h, out)
        return out

    def stats(self):
        m = np.zeros((3, self.ny, self.nx))
        r = np.zeros((6, self.ny, self.nx))
        rc, s = A.stg_lbm_stats(self.h, m, r)
        return dict(rc=rc, step=s.step, n_samples=s.n_samples, mass=s.mass, mass0=s.mass0, mean_sum=m,
                    rey_sum=r, error=A.stg_lbm_last_error(self.h) if rc else "")

    def reset_stats(self):
        """Restart the running statistics at the current step."""
        A.stg_lbm_reset_stats(self.h)

    def info(self):
        i = A.stg_lbm_info(self.h)
        return {k: getattr(i, k) for k, _ in A.stg_info._fields_}

    def device_state(self):
        return A.stg_lbm_device_state(self.h)

    def close(self):
        if getattr(self, "h", None):
            A.stg_lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
