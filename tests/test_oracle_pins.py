"""Pins of the CPU oracle's pointwise pieces against closed forms, invariants
and values printed in the paper.  None of these re-derives a result by
calling the formula under test a second time: each checks a property the
paper or the mathematics fixes independently."""
import math
import os

import numpy as np
import pytest

import oracle as O
from workloads import synthetic_rans_profile, RansProfile

GOLD = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(1234)


def _golden(name):
    vals = {}
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if len(parts) == 2:
            vals[parts[0]] = parts[1]
        else:
            rows.append(parts[0])
    return vals, rows


# ---------------------------------------------------------------- lattice
def test_d3q19_tables_isotropy():
    c, w, opp = O.d3q19()
    assert sorted(map(tuple, c)) == sorted(
        {(a, b, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1) if a * a + b * b + d * d <= 2})
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_array_equal(c[opp], -c)
    cs2 = 1 / 3
    # second and fourth moments of the weights (lattice isotropy)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    np.testing.assert_allclose(M2, cs2 * np.eye(3), atol=1e-15)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(M4, iso, atol=1e-15)


# ---------------------------------------------------------------- draws
def test_splitmix64_published_vector():
    vals, rows = _golden("splitmix64.txt")
    out = O.splitmix64(int(vals["seed"]), len(rows))
    assert [int(v) for v in out] == [int(r) for r in rows]


def test_uniform_draws_range_and_moments():
    u = O.uniform_draws(7, 200000)
    assert u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.002


# ---------------------------------------------------------------- equilibrium / moments
@pytest.mark.parametrize("trial", range(5))
def test_equilibrium_moments_exact(trial):
    rho = rng.uniform(0.8, 1.2)
    u = rng.uniform(-0.1, 0.1, 3)
    c, w, _ = O.d3q19()
    feq = O.equilibrium(rho, u)
    assert abs(feq.sum() - rho) < 1e-14
    np.testing.assert_allclose(c.T @ feq, rho * u, atol=1e-15)
    Pi = np.einsum("ia,ib,i->ab", c, c, feq)
    np.testing.assert_allclose(Pi, rho * (np.eye(3) / 3 + np.outer(u, u)), atol=1e-15)


def test_moments_of_equilibrium_have_no_neq_and_carry_half_force():
    c, w, _ = O.d3q19()
    u = np.array([0.03, -0.01, 0.02])
    F = np.array([1e-3, 2e-3, -1e-3])
    # a state whose bare momentum is rho u - F/2 has macroscopic velocity u (eq. momentum)
    rho = 1.05
    feq = O.equilibrium(rho, u)
    feq_shift = feq - w * (c @ (F / 2)) / (1 / 3)
    r, uu, pi = O.moments(feq_shift, F)
    assert abs(r - rho) < 1e-14
    np.testing.assert_allclose(uu, u, atol=1e-15)


# ---------------------------------------------------------------- regularization
def test_regularized_neq_returns_pi_and_has_no_lower_moments():
    c, w, _ = O.d3q19()
    A = rng.normal(size=(3, 3))
    Pi = 1e-3 * (A + A.T)
    fneq = O.regularized_neq(Pi)
    assert abs(fneq.sum()) < 1e-17
    np.testing.assert_allclose(c.T @ fneq, 0, atol=1e-17)
    Q = np.einsum("ia,ib->iab", c, c) - np.eye(3)[None] / 3
    np.testing.assert_allclose(np.einsum("iab,i->ab", Q, fneq), Pi, atol=1e-17)
    np.testing.assert_allclose(np.einsum("ia,ib,i->ab", c, c, fneq), Pi, atol=1e-17)


# ---------------------------------------------------------------- SGS
def test_tau_eff_limits_and_strain_equation():
    tau0, C = 0.52, 0.01
    assert abs(O.tau_eff(tau0, C, 1.0, 0.0) - tau0) < 1e-15
    assert abs(O.tau_eff(tau0, C, 1.1, 0.0) - tau0) < 1e-15
    Qs = np.linspace(0, 1e-2, 50)
    t = np.array([O.tau_eff(tau0, C, 1.0, q) for q in Qs])
    assert np.all(np.diff(t) > 0)
    # at rho = 1, c = dx = delta = 1: tau_eff = tau0 + 3 C |S| with |S| from eq. (strain)
    for q in [1e-5, 1e-3, 3e-2]:
        S = (-tau0 + math.sqrt(tau0 ** 2 + 18 * math.sqrt(2) * C * q)) / (6 * C)
        nu_eff = (tau0 - 0.5) / 3 + C * S  # eq. (smogrinsky_model) with nu0 from eq. (lbe-nu)
        assert abs(O.tau_eff(tau0, C, 1.0, q) - (3 * nu_eff + 0.5)) < 1e-14
    # C = 0 switches the model off
    assert O.tau_eff(0.6, 0.0, 1.0, 0.5) == pytest.approx(0.6, abs=1e-15)


def test_collision_conserves_mass_and_momentum():
    c, w, _ = O.d3q19()
    for coll in ["regularized", "bgk"]:
        for F in [(0, 0, 0), (1e-4, -2e-4, 5e-5)]:
            f = w * (1 + 0.05 * rng.normal(size=19))
            out, rho, u = O.collide(f, 0.55, 0.01, F, coll)
            assert abs(out.sum() - f.sum()) < 1e-15
            np.testing.assert_allclose(c.T @ out, c.T @ f + np.array(F), atol=1e-16)


def test_collision_tau_one_gives_equilibrium():
    c, w, _ = O.d3q19()
    f = w * (1 + 0.05 * rng.normal(size=19))
    out, rho, u = O.collide(f, 1.0, 0.0, (0, 0, 0), "regularized")
    np.testing.assert_allclose(out, O.equilibrium(rho, u), atol=1e-16)
    out2, _, _ = O.collide(f, 1.0, 0.0, (0, 0, 0), "bgk")
    np.testing.assert_allclose(out2, out, atol=1e-16)


def test_regularized_collision_keeps_only_second_order_neq():
    # the post-collision non-equilibrium part is (1 - 1/tau) times the
    # projection on Q_i, whatever higher-order content the input carries
    c, w, _ = O.d3q19()
    rho0, u0 = 1.02, np.array([0.02, 0.01, -0.03])
    feq = O.equilibrium(rho0, u0)
    ghost = w * rng.normal(size=19) * 1e-3
    # remove the parts the projection keeps (orders 0, 1, 2) from the ghost
    H = np.concatenate([np.ones((19, 1)), c, np.einsum("ia,ib->iab", c, c).reshape(19, 9)], axis=1)
    ghost -= H @ np.linalg.lstsq(H, ghost, rcond=None)[0]
    out_plain, _, _ = O.collide(feq, 0.6, 0.0)
    out_ghost, _, _ = O.collide(feq + ghost, 0.6, 0.0)
    np.testing.assert_allclose(out_ghost, out_plain, atol=1e-16)
    np.testing.assert_allclose(out_plain, feq, atol=1e-16)


# ---------------------------------------------------------------- inlet / outlet
def test_zou_he_density_exact_for_equilibrium():
    for _ in range(5):
        rho0 = rng.uniform(0.9, 1.1)
        u = rng.uniform(-0.05, 0.05, 3)
        feq = O.equilibrium(rho0, u)
        assert abs(O.zou_he_density(feq, u[0]) - rho0) < 1e-14


def test_inlet_reconstruction_fixed_point_and_moments():
    c, w, _ = O.d3q19()
    rho0, u = 1.01, np.array([0.04, 0.005, -0.003])
    A = rng.normal(size=(3, 3))
    Pi = 1e-4 * (A + A.T)
    f = O.equilibrium(rho0, u) + O.regularized_neq(Pi)
    f_known = f.copy()
    f_known[c[:, 0] > 0] = 7.0  # unknowns must not matter
    out = O.inlet_reconstruct(f_known, u)
    # rebuilt density/velocity are the prescribed ones; a regularized state is a fixed point
    assert abs(out.sum() - O.zou_he_density(f, u[0])) < 1e-14
    np.testing.assert_allclose(c.T @ out / out.sum(), u, atol=1e-15)
    # a regularized state is rebuilt exactly (its non-equilibrium part is even in c)
    f_nan = f.copy()
    f_nan[c[:, 0] > 0] = np.nan
    np.testing.assert_allclose(O.inlet_reconstruct(f_nan, u), f, atol=1e-15)
    assert abs(O.zou_he_density(f, u[0]) - rho0) < 1e-14


def test_outlet_uniform_flow_fixed_point():
    c, w, _ = O.d3q19()
    U = np.array([0.03, 0.0, 0.0])
    feq = O.equilibrium(1.0, U)
    fk = feq.copy()
    fk[c[:, 0] < 0] = np.nan
    out = O.outlet_reconstruct(fk, U)
    np.testing.assert_allclose(out, feq, atol=1e-16)


# ---------------------------------------------------------------- STG setup pieces
def test_cholesky_reproduces_stress():
    for _ in range(10):
        A = rng.normal(size=(3, 3))
        R = A @ A.T + 0.1 * np.eye(3)
        R6 = np.array([R[0, 0], R[1, 1], R[2, 2], R[1, 0], R[2, 0], R[2, 1]])
        a6 = O.cholesky(R6)
        L = np.array([[a6[0], 0, 0], [a6[1], a6[2], 0], [a6[3], a6[4], a6[5]]])
        np.testing.assert_allclose(L @ L.T, R, atol=1e-13)
        assert np.all(np.diag(L) > 0)
    # wall limit: R = 0 gives a = 0 with no NaN
    np.testing.assert_array_equal(O.cholesky(np.zeros(6)), 0.0)


def test_spectrum_peak_and_kolmogorov_slope():
    le = 10.0
    ke = 2 * math.pi / le
    ks = ke * np.linspace(0.5, 2.0, 3001)
    E = np.array([O.spectrum(k, le, 0.0, 0.0) for k in ks])
    # the von Karman part peaks exactly at k = k_e
    assert abs(ks[np.argmax(E)] / ke - 1) < 1e-3
    # far above k_e the spectrum follows the -5/3 law (Sec. III: "-5/3 energy spectrum")
    k1, k2 = 1e3 * ke, 1e4 * ke
    slope = math.log(O.spectrum(k2, le, 0, 0) / O.spectrum(k1, le, 0, 0)) / math.log(k2 / k1)
    assert abs(slope + 5 / 3) < 1e-4
    # the viscous and cut-off factors only damp, and do nothing below 0.9 k_cut
    lcut = 2.0
    kcut = 2 * math.pi / lcut
    assert O.spectrum(0.8 * kcut, le, 0, lcut) == pytest.approx(O.spectrum(0.8 * kcut, le, 0, 0), rel=1e-15)
    assert O.spectrum(1.2 * kcut, le, 0, lcut) < O.spectrum(1.2 * kcut, le, 0, 0)
    leta = 0.1
    keta = 2 * math.pi / leta
    assert O.spectrum(keta / 12, le, leta, 0) == pytest.approx(O.spectrum(keta / 12, le, 0, 0) * math.exp(-1), rel=1e-14)


def test_unit_conversion_paper_example():
    vals, _ = _golden("unit_conversion.txt")
    tau0, ny = float(vals["tau0"]), int(vals["ny"])
    prof = RansProfile(y_c=np.array([0.5, 1.5]), U=np.array([float(vals["U_max"])] * 2), k=np.zeros(2),
                       eps=np.ones(2), R=np.zeros((2, 6)), U_bulk=15.37, nu_phys=float(vals["nu_phys"]),
                       h_phys=float(vals["h_phys"]), re_tau=180.0)
    cx, ct = O.unit_scales(prof, tau0, ny, 0.0)
    tol = float(vals["rel_tol"])
    assert cx == pytest.approx(float(vals["c_x"]), rel=1e-15)
    assert ct == pytest.approx(float(vals["c_t"]), rel=tol)
    ma = float(vals["U_max"]) * ct / cx / math.sqrt(1 / 3)
    assert ma == pytest.approx(float(vals["mach"]), rel=tol)
    # Mach-target route maps U_max to mach * c_s exactly
    cx2, ct2 = O.unit_scales(prof, tau0, ny, 0.0516)
    assert float(vals["U_max"]) * ct2 / cx2 == pytest.approx(0.0516 * math.sqrt(1 / 3), rel=1e-15)


def test_filter_impulse_response_and_dc_gain():
    a = math.exp(-1 / 4.0)
    uf = np.zeros(1)
    O.filter_update(True, a, np.zeros(1), uf)
    seq = []
    for n in range(6):
        O.filter_update(False, a, np.array([1.0 if n == 0 else 0.0]), uf)
        seq.append(uf[0])
    np.testing.assert_allclose(seq, (1 - a) * a ** np.arange(6), rtol=1e-15)
    # unit gain at zero frequency; a = 0 is the identity
    uf = np.array([0.0])
    for _ in range(400):
        O.filter_update(False, a, np.array([2.5]), uf)
    assert uf[0] == pytest.approx(2.5, rel=1e-12)
    uf = np.array([9.0])
    O.filter_update(False, 0.0, np.array([1.25]), uf)
    assert uf[0] == 1.25
    # sinusoid gain |H(w)| = (1-a)/|1 - a e^{-iw}|
    w = 0.3
    uf = np.zeros(1)
    out = []
    for n in range(3000):
        O.filter_update(n == 0, a, np.array([math.cos(w * n)]), uf)
        out.append(uf[0])
    amp = np.abs(np.array(out[2000:])).max()
    assert amp == pytest.approx((1 - a) / abs(1 - a * np.exp(-1j * w)), rel=2e-3)


def test_f16_decoder():
    vals = np.array([0.0, -0.0, 1.0, -2.5, 6.1e-5, 3e-7, 65504.0, 0.333], dtype=np.float16)
    for v in vals:
        assert O.f16_to_double(int(v.view(np.uint16))) == float(v)


def test_synthetic_profile_is_realisable():
    for re in (180.0, 395.0):
        for n in (48, 96):
            p = synthetic_rans_profile(re, n)
            assert np.all(np.diff(p.y_c) > 0)
            for R6 in p.R:
                R = np.array([[R6[0], R6[3], R6[4]], [R6[3], R6[1], R6[5]], [R6[4], R6[5], R6[2]]])
                assert np.linalg.eigvalsh(R).min() > 0
            assert np.all(p.eps > 0) and np.all(p.k > 0)
