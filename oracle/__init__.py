"""ctypes front end of the CPU FP64 oracle.

TEST INFRASTRUCTURE ONLY: only the test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  It never imports
the CUDA library and the CUDA library never imports it.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None

c_double_p = C.POINTER(C.c_double)
c_int32_p = C.POINTER(C.c_int32)
c_int64_p = C.POINTER(C.c_int64)
c_uint64_p = C.POINTER(C.c_uint64)


class Domain(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("bc_x", C.c_int32), ("bc_y", C.c_int32), ("collision", C.c_int32),
                ("stats_every", C.c_int32), ("pad0", C.c_int32),
                ("tau0", C.c_double), ("c_smag", C.c_double), ("force", C.c_double * 3),
                ("sponge_len", C.c_double), ("sponge_K", C.c_double), ("sponge_p", C.c_double)]


class Rans(C.Structure):
    _fields_ = [("n_fv", C.c_int32), ("pad0", C.c_int32),
                ("y_c", c_double_p), ("U", c_double_p), ("k", c_double_p), ("eps", c_double_p),
                ("R", c_double_p),
                ("U_bulk", C.c_double), ("nu_phys", C.c_double), ("h_phys", C.c_double),
                ("mach_target", C.c_double)]


class StgParams(C.Structure):
    _fields_ = [("n_modes", C.c_int32), ("pad0", C.c_int32),
                ("C_l", C.c_double), ("alpha", C.c_double), ("T_filter", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "orc_d3q19": (None, [c_int32_p, c_double_p, c_int32_p]),
            "orc_splitmix64": (None, [C.c_uint64, C.c_int32, c_uint64_p]),
            "orc_uniform_draws": (None, [C.c_uint64, C.c_int32, c_double_p]),
            "orc_equilibrium": (None, [C.c_double, c_double_p, c_double_p]),
            "orc_moments": (None, [c_double_p, c_double_p, c_double_p, c_double_p, c_double_p]),
            "orc_tau_eff": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_double]),
            "orc_regularized_neq": (None, [c_double_p, c_double_p]),
            "orc_collide": (None, [C.POINTER(Domain), c_double_p, c_double_p, c_double_p, c_double_p]),
            "orc_sponge_factor": (C.c_double, [C.POINTER(Domain), C.c_int32]),
            "orc_zou_he_density": (C.c_double, [c_double_p, C.c_double]),
            "orc_inlet_reconstruct": (None, [c_double_p, c_double_p, c_double_p]),
            "orc_outlet_reconstruct": (None, [c_double_p, c_double_p, c_double_p]),
            "orc_cholesky": (None, [c_double_p, c_double_p]),
            "orc_spectrum": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_double]),
            "orc_unit_scales": (None, [C.POINTER(Rans), C.c_double, C.c_int32, c_double_p, c_double_p]),
            "orc_filter_update": (None, [C.c_int32, C.c_double, c_double_p, c_double_p, C.c_int32]),
            "orc_f16_to_double": (C.c_double, [C.c_uint16]),
            "orc_cell_update": (None, [C.POINTER(Domain), C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                       C.c_int32, c_double_p, c_double_p]),
            "orc_sim_create": (C.c_int32, [C.POINTER(Domain), C.POINTER(Rans), C.POINTER(StgParams),
                                           C.c_uint64, C.POINTER(C.c_void_p)]),
            "orc_sim_destroy": (None, [C.c_void_p]),
            "orc_sim_set_pops": (None, [C.c_void_p, c_double_p]),
            "orc_sim_get_pops": (None, [C.c_void_p, c_double_p]),
            "orc_sim_step": (None, [C.c_void_p, C.c_int32]),
            "orc_sim_time": (C.c_int64, [C.c_void_p]),
            "orc_sim_mass": (C.c_double, [C.c_void_p]),
            "orc_sim_get_inlet": (None, [C.c_void_p, c_double_p]),
            "orc_sim_get_stats": (None, [C.c_void_p, c_double_p, c_double_p, c_int64_p]),
            "orc_sim_n_modes": (C.c_int32, [C.c_void_p]),
            "orc_sim_scalars": (None, [C.c_void_p, c_double_p]),
            "orc_sim_tables": (None, [C.c_void_p] + [c_double_p] * 8),
            "orc_sim_stg_raw": (None, [C.c_void_p, C.c_double, C.c_int32, C.c_int32, c_double_p]),
            "orc_threads": (C.c_int32, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(c_double_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------
# pointwise helpers
# ----------------------------------------------------------------------------
def d3q19():
    c = np.zeros(57, np.int32)
    w = np.zeros(19)
    o = np.zeros(19, np.int32)
    lib().orc_d3q19(c.ctypes.data_as(c_int32_p), _dp(w), o.ctypes.data_as(c_int32_p))
    return c.reshape(19, 3), w, o


def splitmix64(seed, n):
    out = np.zeros(n, np.uint64)
    lib().orc_splitmix64(seed, n, out.ctypes.data_as(c_uint64_p))
    return out


def uniform_draws(seed, n):
    out = np.zeros(n)
    lib().orc_uniform_draws(seed, n, _dp(out))
    return out


def equilibrium(rho, u):
    u = _f64(u)
    out = np.zeros(19)
    lib().orc_equilibrium(rho, _dp(u), _dp(out))
    return out


def moments(f, F=(0.0, 0.0, 0.0)):
    f = _f64(f)
    F = _f64(F)
    rho = np.zeros(1)
    u = np.zeros(3)
    pi = np.zeros(9)
    lib().orc_moments(_dp(f), _dp(F), _dp(rho), _dp(u), _dp(pi))
    return rho[0], u, pi.reshape(3, 3)


def tau_eff(tau0, C_, rho, Q_half):
    return lib().orc_tau_eff(tau0, C_, rho, Q_half)


def regularized_neq(pi):
    pi = _f64(pi).reshape(9)
    out = np.zeros(19)
    lib().orc_regularized_neq(_dp(pi), _dp(out))
    return out


def make_domain(nx, ny, nz, tau0=0.52, c_smag=0.01, force=(0.0, 0.0, 0.0), bc_x="stg",
                bc_y="walls", collision="regularized", stats_every=0, sponge=(0.0, 1000.0, 3.0)):
    """sponge = (length before the outlet column, K, p) of eq. (sponge_visco); length 0: off."""
    d = Domain()
    d.sponge_len, d.sponge_K, d.sponge_p = sponge
    d.nx, d.ny, d.nz = nx, ny, nz
    d.bc_x = {"stg": 0, "periodic": 1}[bc_x]
    d.bc_y = {"walls": 0, "periodic": 1}[bc_y]
    d.collision = {"regularized": 0, "bgk": 1}[collision]
    d.stats_every = stats_every
    d.tau0, d.c_smag = tau0, c_smag
    d.force = (C.c_double * 3)(*force)
    return d


def collide(f, tau0=0.52, c_smag=0.01, force=(0.0, 0.0, 0.0), collision="regularized"):
    d = make_domain(1, 1, 1, tau0, c_smag, force, "periodic", "periodic", collision)
    f = _f64(f)
    out = np.zeros(19)
    rho = np.zeros(1)
    u = np.zeros(3)
    lib().orc_collide(C.byref(d), _dp(f), _dp(out), _dp(rho), _dp(u))
    return out, rho[0], u


def sponge_factor(domain, x):
    """nu_sponge / nu_eff at column x, eq. (sponge_visco)."""
    return lib().orc_sponge_factor(C.byref(domain), int(x))


def zou_he_density(f, ux):
    return lib().orc_zou_he_density(_dp(_f64(f)), ux)


def inlet_reconstruct(f, u_bc):
    out = np.zeros(19)
    lib().orc_inlet_reconstruct(_dp(_f64(f)), _dp(_f64(u_bc)), _dp(out))
    return out


def outlet_reconstruct(f, u_out):
    out = np.zeros(19)
    lib().orc_outlet_reconstruct(_dp(_f64(f)), _dp(_f64(u_out)), _dp(out))
    return out


def cholesky(R6):
    a = np.zeros(6)
    lib().orc_cholesky(_dp(_f64(R6)), _dp(a))
    return a


def spectrum(k, l_e, l_eta, l_cut):
    return lib().orc_spectrum(k, l_e, l_eta, l_cut)


def filter_update(first, a, u_raw, u_f):
    u_raw = _f64(u_raw)
    lib().orc_filter_update(int(first), a, _dp(u_raw), _dp(u_f), u_raw.size)
    return u_f


def f16_to_double(bits):
    return lib().orc_f16_to_double(int(bits))


class _RansHolder:
    """Keeps the numpy arrays behind an ``Rans`` struct alive."""

    def __init__(self, prof, mach_target):
        self.arrays = [_f64(prof.y_c), _f64(prof.U), _f64(prof.k), _f64(prof.eps),
                       _f64(prof.R).reshape(-1)]
        r = Rans()
        r.n_fv = prof.n_fv
        r.y_c, r.U, r.k, r.eps, r.R = [_dp(a) for a in self.arrays]
        r.U_bulk, r.nu_phys, r.h_phys = prof.U_bulk, prof.nu_phys, prof.h_phys
        r.mach_target = mach_target
        self.struct = r


def unit_scales(prof, tau0, ny, mach_target):
    h = _RansHolder(prof, mach_target)
    cx = np.zeros(1)
    ct = np.zeros(1)
    lib().orc_unit_scales(C.byref(h.struct), tau0, ny, _dp(cx), _dp(ct))
    return cx[0], ct[0]


def cell_update(domain, src, x, y, z, u_bc=(0.0, 0.0, 0.0), shifted=False):
    """One cell's post-step populations from a stored lattice.

    ``src`` is float64 (f), float32 (f, or f_i - w_i with ``shifted``), or
    uint16 (binary16 bits of f_i - w_i)."""
    if src.dtype == np.float64:
        t = 0
    elif src.dtype == np.float32:
        t = 3 if shifted else 1
    elif src.dtype == np.uint16:
        t = 2
    else:
        raise TypeError(src.dtype)
    assert src.flags.c_contiguous
    out = np.zeros(19)
    ub = _f64(u_bc)
    lib().orc_cell_update(C.byref(domain), t, C.c_void_p(src.ctypes.data), x, y, z, _dp(ub), _dp(out))
    return out


# ----------------------------------------------------------------------------
# simulation
# ----------------------------------------------------------------------------
class Sim:
    """FP64 two-lattice STG-LBM simulation (the oracle)."""

    def __init__(self, nx, ny, nz, tau0=0.52, c_smag=0.01, force=(0.0, 0.0, 0.0), bc_x="stg",
                 bc_y="walls", collision="regularized", stats_every=0, profile=None,
                 n_modes=100, C_l=3.0, alpha=0.01, t_filter=0.0, mach_target=0.0516, seed=0,
                 sponge=(0.0, 1000.0, 3.0)):
        self.domain = make_domain(nx, ny, nz, tau0, c_smag, force, bc_x, bc_y, collision, stats_every, sponge)
        self.nx, self.ny, self.nz = nx, ny, nz
        self._rans = _RansHolder(profile, mach_target) if profile is not None else None
        p = StgParams()
        p.n_modes, p.C_l, p.alpha, p.T_filter = n_modes, C_l, alpha, t_filter
        self._p = p
        h = C.c_void_p()
        rc = lib().orc_sim_create(C.byref(self.domain),
                                  C.byref(self._rans.struct) if self._rans else None,
                                  C.byref(p), seed, C.byref(h))
        if rc != 0:
            raise ValueError(f"orc_sim_create failed ({rc})")
        self.h = h

    @classmethod
    def from_case(cls, case, **kw):
        args = dict(tau0=case.tau0, c_smag=case.c_smag, force=case.force, bc_x=case.bc_x,
                    bc_y=case.bc_y, collision=case.collision, stats_every=case.stats_every,
                    profile=case.profile() if case.bc_x == "stg" else None, n_modes=case.n_modes,
                    t_filter=case.t_filter, mach_target=case.mach_target, seed=case.seed,
                    sponge=(case.sponge_len, case.sponge_K, case.sponge_p))
        args.update(kw)
        return cls(case.nx, case.ny, case.nz, **args)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_sim_destroy(self.h)
            self.h = None

    @property
    def shape(self):
        return (19, self.nz, self.ny, self.nx)

    def set_pops(self, f):
        f = _f64(f)
        assert f.shape == self.shape
        lib().orc_sim_set_pops(self.h, _dp(f))

    def pops(self):
        f = np.zeros(self.shape)
        lib().orc_sim_get_pops(self.h, _dp(f))
        return f

    def step(self, n=1):
        lib().orc_sim_step(self.h, n)

    @property
    def time(self):
        return lib().orc_sim_time(self.h)

    @property
    def mass(self):
        return lib().orc_sim_mass(self.h)

    def inlet(self):
        u = np.zeros((3, self.nz, self.ny))
        lib().orc_sim_get_inlet(self.h, _dp(u))
        return u

    def stats(self):
        m = np.zeros((3, self.ny, self.nx))
        r = np.zeros((6, self.ny, self.nx))
        n = np.zeros(1, np.int64)
        lib().orc_sim_get_stats(self.h, _dp(m), _dp(r), n.ctypes.data_as(c_int64_p))
        return m, r, int(n[0])

    def scalars(self):
        o = np.zeros(8)
        lib().orc_sim_scalars(self.h, _dp(o))
        keys = ["c_x", "c_t", "U_b", "max_le", "k_min", "k_max", "n_modes", "a_filter"]
        return dict(zip(keys, o))

    def tables(self):
        ny = self.ny
        N = lib().orc_sim_n_modes(self.h)
        t = dict(u_int=np.zeros(ny), a6=np.zeros((ny, 6)), l_e=np.zeros(ny), q=np.zeros((ny, N)),
                 kn=np.zeros(N), d=np.zeros((N, 3)), sigma=np.zeros((N, 3)), phi=np.zeros(N))
        lib().orc_sim_tables(self.h, *[_dp(t[k]) for k in ["u_int", "a6", "l_e", "q", "kn", "d", "sigma", "phi"]])
        return t

    def stg_raw(self, t, j, k):
        u = np.zeros(3)
        lib().orc_sim_stg_raw(self.h, float(t), j, k, _dp(u))
        return u


def threads():
    return int(lib().orc_threads())


__all__ = [n for n in dir() if not n.startswith("_")]
