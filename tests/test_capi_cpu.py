"""CPU-side checks of the C ABI: the library loads, exports every function the
header declares, rejects bad arguments before touching the GPU, and draws the
same random mode parameters as the oracle (bit for bit)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2205_02774_gb300 import build
    build()
    from paper_2205_02774_gb300 import capi
    capi.lib()
    return capi


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "stg_lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stg_\w+)\s*\(", text)))


def test_header_symbols_exported(capi):
    names = _declared_functions()
    assert "stg_lbm_create" in names and "stg_lbm_step" in names and "stg_lbm_stats" in names
    assert "stg_lbm_destroy" in names
    L = C.CDLL(capi.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(capi._SIGNATURES) == set(names)


def test_version(capi):
    assert "sm_103a" in capi.stg_lbm_version()


def test_mode_draws_match_oracle(capi):
    import oracle as O
    for seed in (0, 1, 12345, 2 ** 63 + 7):
        a = capi.stg_mode_draws(seed, 250)
        b = O.uniform_draws(seed, 1000)
        np.testing.assert_array_equal(a, b)


def _domain(capi, **kw):
    d = capi.stg_domain()
    d.nx, d.ny, d.nz = kw.get("nx", 8), kw.get("ny", 8), kw.get("nz", 8)
    d.storage = kw.get("storage", 0)
    d.collision = kw.get("collision", 0)
    d.bc_x = kw.get("bc_x", capi.STG_BC_X_PERIODIC)
    d.bc_y = kw.get("bc_y", 0)
    d.tau0 = kw.get("tau0", 0.6)
    d.c_smag = kw.get("c_smag", 0.01)
    d.streaming = kw.get("streaming", 0)
    return d


@pytest.mark.parametrize("kw,msg", [
    (dict(nx=0), "sizes"),
    (dict(tau0=0.5), "tau0"),
    (dict(storage=7), "storage"),
    (dict(collision=3), "collision"),
    (dict(c_smag=-1.0), "c_smag"),
    (dict(bc_x=0, nx=2), "nx >= 3"),
    (dict(bc_x=0), "RANS profile"),
    (dict(nx=2048, ny=2048, nz=1024), "2^31"),
    (dict(streaming=5), "bad streaming"),
    (dict(streaming=1, nx=7), "in-place streaming"),        # odd nx
    (dict(streaming=1, nx=2), "in-place streaming"),        # nx < 4
    (dict(streaming=1, nx=2048, ny=1024, nz=128), "in-place streaming"),  # 19 nx ny nz >= 2^32
])
def test_create_rejects_bad_arguments(capi, kw, msg):
    d = _domain(capi, **kw)
    with pytest.raises(capi.StgError) as e:
        capi.stg_lbm_create(d, None, None, 0)
    assert e.value.code == capi.STG_ERR_INVALID
    assert msg in str(e.value)


def test_create_rejects_bad_profile(capi):
    from workloads import synthetic_rans_profile
    p = synthetic_rans_profile(180.0, 16)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (p.y_c, p.U, p.k, p.eps)]
    R = np.ascontiguousarray(p.R, dtype=np.float64).reshape(-1)
    r = capi.stg_rans_profile()
    r.n_fv = 16
    r.y_c, r.U, r.k, r.eps = [a.ctypes.data_as(capi.c_double_p) for a in arrs]
    r.R = R.ctypes.data_as(capi.c_double_p)
    r.U_bulk, r.nu_phys, r.h_phys, r.mach_target = p.U_bulk, p.nu_phys, p.h_phys, 0.05
    prm = capi.stg_params()
    prm.n_modes, prm.C_l, prm.alpha, prm.T_filter = 10, 3.0, 0.01, 0.0
    d = _domain(capi, bc_x=0)
    arrs[0][3] = arrs[0][2]  # not strictly increasing
    with pytest.raises(capi.StgError) as e:
        capi.stg_lbm_create(d, r, prm, 0)
    assert e.value.code == capi.STG_ERR_INVALID and "y_c" in str(e.value)


@pytest.mark.parametrize("kw", [dict(storage=2), dict(streaming=1), dict(storage=2, streaming=1, nx=4)])
def test_create_accepts_stochastic_rounding_and_in_place(capi, kw):
    """The binary16 storage by stochastic rounding and the in-place scheme pass
    the argument checks (without a GPU the call then fails in CUDA, not in
    validation)."""
    d = _domain(capi, **kw)
    try:
        h = capi.stg_lbm_create(d, None, None, 0)
    except capi.StgError as e:
        assert e.code == capi.STG_ERR_CUDA, str(e)
    else:
        capi.stg_lbm_destroy(h)


def test_reset_stats_rejects_null(capi):
    assert capi.lib().stg_lbm_reset_stats(None) == capi.STG_ERR_INVALID
