"""Statistical and closed-form pins of the oracle's synthetic turbulence
generator (Sec. III.A): over independent seeds the fluctuation has zero mean
and the prescribed Reynolds stress, the random directions are uniform on the
sphere with sigma normal to d, the amplitudes q^n sum to one, and the
interpolation and length scales reduce to their definitions in special cases."""
import math

import numpy as np
import pytest

import oracle as O
from workloads import RansProfile, synthetic_rans_profile, tanh_grid

NY = 16
NODES = [(0, 0), (3, 0), (8, 0), (12, 0)]


@pytest.fixture(scope="module")
def samples():
    prof = synthetic_rans_profile(180.0, 48)
    seeds = range(20000)
    out = np.zeros((len(seeds), len(NODES), 3))
    for s in seeds:
        sim = O.Sim(3, NY, 1, profile=prof, n_modes=100, t_filter=0.0, seed=s)
        for m, (j, k) in enumerate(NODES):
            out[s, m] = sim.stg_raw(37.0, j, k)
    ref = O.Sim(3, NY, 1, profile=prof, n_modes=100, t_filter=0.0, seed=0)
    return out, ref.tables()


def test_stg_fluctuation_mean_is_zero(samples):
    u, tab = samples
    n = u.shape[0]
    for m in range(len(NODES)):
        se = u[:, m].std(0) / math.sqrt(n)
        assert np.all(np.abs(u[:, m].mean(0)) < 4.5 * se + 1e-30)


def test_stg_reproduces_reynolds_stress(samples):
    """<u'u'^T> over seeds equals a a^T = R (Cholesky of the interpolated,
    lattice-scaled stress): the sqrt(6), the unit sigma normal to d and the
    normalisation sum q^n = 1 together give <v'v'^T> = I."""
    u, tab = samples
    n = u.shape[0]
    for m, (j, _) in enumerate(NODES):
        a6 = tab["a6"][j]
        L = np.array([[a6[0], 0, 0], [a6[1], a6[2], 0], [a6[3], a6[4], a6[5]]])
        R = L @ L.T
        for a in range(3):
            for b in range(a, 3):
                prod = u[:, m, a] * u[:, m, b]
                se = prod.std() / math.sqrt(n)
                assert abs(prod.mean() - R[a, b]) < 4.5 * se, (j, a, b, prod.mean(), R[a, b], se)


def test_mode_directions_uniform_and_orthogonal():
    prof = synthetic_rans_profile(180.0, 48)
    D, S = [], []
    for s in range(200):
        t = O.Sim(3, 8, 1, profile=prof, n_modes=100, seed=s).tables()
        D.append(t["d"])
        S.append(t["sigma"])
        np.testing.assert_allclose(np.linalg.norm(t["d"], axis=1), 1, atol=1e-14)
        np.testing.assert_allclose(np.linalg.norm(t["sigma"], axis=1), 1, atol=1e-14)
        np.testing.assert_allclose(np.einsum("na,na->n", t["d"], t["sigma"]), 0, atol=1e-14)
        assert t["phi"].min() >= 0 and t["phi"].max() < 2 * math.pi
    D = np.concatenate(D)
    S = np.concatenate(S)
    n = D.shape[0]
    assert np.all(np.abs(D.mean(0)) < 4.5 * math.sqrt(1 / 3 / n))
    np.testing.assert_allclose(D.T @ D / n, np.eye(3) / 3, atol=0.01)
    np.testing.assert_allclose(S.T @ S / n, np.eye(3) / 3, atol=0.01)


def test_amplitudes_normalised_and_wavenumbers_geometric():
    prof = synthetic_rans_profile(180.0, 48)
    sim = O.Sim(3, 32, 1, profile=prof, n_modes=100, seed=0)
    t = sim.tables()
    sc = sim.scalars()
    np.testing.assert_allclose(t["q"].sum(1), 1.0, atol=1e-13)
    assert t["q"].min() >= 0
    kn = t["kn"]
    assert kn[0] == pytest.approx(sc["k_min"], rel=1e-15)
    assert kn[-1] == pytest.approx(sc["k_max"], rel=1e-13)
    r = kn[1:] / kn[:-1]
    np.testing.assert_allclose(r, r[0], rtol=1e-12)
    assert sc["k_min"] == pytest.approx(math.pi / sc["max_le"], rel=1e-15)
    # lattice spacing 1 in eq. (lcut): l_cut = 2, so k_max = 1.5 * 2 pi / 2
    assert sc["k_max"] == pytest.approx(1.5 * math.pi, rel=1e-15)
    # mode count from eq. (Nmode) when none is configured
    sim2 = O.Sim(3, 32, 1, profile=prof, n_modes=0, alpha=0.01, seed=0)
    N = int(sim2.scalars()["n_modes"])
    assert N == math.ceil(math.log(sc["k_max"] / sc["k_min"]) / math.log(1.01) + 1)


def _profile(U, k, eps, R):
    n = 48
    faces = tanh_grid(n)
    y_c = 0.5 * (faces[1:] + faces[:-1])
    f = lambda v: np.broadcast_to(v(y_c) if callable(v) else v, (n,)).astype(float).copy()
    Rm = np.zeros((n, 6))
    for c in range(6):
        Rm[:, c] = f(R[c])
    return RansProfile(y_c=y_c, U=f(U), k=f(k), eps=f(eps), R=Rm, U_bulk=1.0, nu_phys=1e-3,
                       h_phys=1.0, re_tau=180.0), y_c


def test_interpolation_reproduces_piecewise_linear_profile():
    tent = lambda y: 10.0 * np.minimum(y, 2 - y)
    prof, y_c = _profile(tent, 1.0, 1.0, [lambda y: 1 + y, 0.5, 0.5, 0.0, 0.0, 0.0])
    ny = 40
    sim = O.Sim(3, ny, 1, profile=prof, n_modes=8, mach_target=0.05, seed=0)
    sc = sim.scalars()
    su = sc["c_t"] / sc["c_x"]
    t = sim.tables()
    y = (np.arange(ny) + 0.5) * sc["c_x"]
    inside = (y >= y_c[0]) & (y <= y_c[23])  # below the centre interval: exactly linear
    np.testing.assert_allclose(t["u_int"][inside], tent(y[inside]) * su, rtol=1e-13)
    # R11 = 1 + y is linear over the whole FV range: a11^2 = R11 su^2
    mid = (y >= y_c[0]) & (y <= y_c[-1])
    np.testing.assert_allclose(t["a6"][mid, 0] ** 2, (1 + y[mid]) * su ** 2, rtol=1e-12)


def test_energy_length_is_wall_limited_when_turbulence_is_large():
    prof, _ = _profile(1.0, 1e6, 1.0, [1.0, 1.0, 1.0, 0, 0, 0])
    ny = 20
    sim = O.Sim(3, ny, 1, profile=prof, n_modes=8, mach_target=0.05, seed=0)
    j = np.arange(ny)
    # l_e = min(2 d_w, C_l l_t) -> 2 d_w, in lattice units d_w = min(j + 1/2, ny - j - 1/2)
    np.testing.assert_allclose(sim.tables()["l_e"], 2 * np.minimum(j + 0.5, ny - j - 0.5), rtol=1e-12)


# ---------------------------------------------------------------------------
# Time and space structure of the generator, eqs. (aux_vec), (psu), (dn).
#
# For one mode n the phase at inlet node (y, z) and step t is
#     a_n = -c0 d_x t + k^n (d_y y + d_z z) + phi^n,   c0 = 2 pi U_b / max l_e,
# because eq. (psu) scales the streamwise pseudo-coordinate by 2 pi/(k^n max l_e)
# and x = 0 at the inlet.  Over the random draws (phi uniform, sigma uniform on
# the circle normal to d, d uniform on the sphere, modes independent):
#   E_phi[cos a cos(a + D)] = cos(D) / 2,   E_eta[sigma sigma^T] = (I - d d^T) / 2,
# so for two nodes and two times, with w_n = (-c0 tau, k^n dy, k^n dz),
#   <v'(y1, z, t) v'(y2, z + dz, t + tau)^T>
#       = 3/2 sum_n sqrt(q^n(y1) q^n(y2)) E_d[(I - d d^T) cos(w_n . d)].
# The sphere average of cos(w . d) is j0(r) = sin(r)/r, r = |w|, and two
# derivatives in w give E_d[(I - d d^T) cos(w . d)] = A(r) I + B(r) w w^T / r^2
# with A = j0 + j0'/r and B = -j0 - 3 j0'/r (j0'' = -j0 - 2 j0'/r).  At equal
# positions the trace is 3 sin(c0 tau)/(c0 tau).  The xz (and xy) entries are
# odd in U_b: they fix the direction in which the pseudo-position advects, the
# spatial entries fix k^n d . x over y and z, and q^n(y) weights every entry.
# ---------------------------------------------------------------------------
CORR_NY = 16
CORR_T0 = 37.0
CORR_Z0 = 4
# (j1, j2, dz, tau): same node at several lags, span and wall-normal separations
CORR_CASES = [(5, 5, 0, 0.0), (5, 5, 0, 200.0), (5, 5, 0, 500.0), (5, 5, 0, 1000.0),
              (5, 5, 1, 0.0), (5, 5, 1, 150.0), (5, 5, 2, 100.0), (3, 3, 1, 150.0),
              (5, 7, 0, 0.0), (5, 7, 0, 120.0), (8, 9, 1, 80.0)]


def _sphere_tensor(r):
    """A(r), B(r) of E_d[(I - d d^T) cos(w . d)] = A I + B w w^T / |w|^2."""
    r = np.asarray(r, dtype=np.float64)
    big = r > 1e-3
    rs = np.where(big, r, 1.0)
    j0 = np.sin(rs) / rs
    jp_r = (rs * np.cos(rs) - np.sin(rs)) / rs ** 3  # j0'(r) / r
    A = np.where(big, j0 + jp_r, 2.0 / 3.0 - r * r / 15.0)
    B = np.where(big, -j0 - 3.0 * jp_r, -r * r / 15.0)
    return A, B


def _corr_closed_form(q1, q2, kn, c0, dy, dz, tau):
    w = np.stack([np.full_like(kn, -c0 * tau), kn * dy, kn * dz], axis=1)
    r = np.linalg.norm(w, axis=1)
    A, B = _sphere_tensor(r)
    wh = np.where(r[:, None] > 0, w / np.where(r > 0, r, 1.0)[:, None], 0.0)
    amp = 1.5 * np.sqrt(q1 * q2)
    return (np.einsum("n,n->", amp, A) * np.eye(3)
            + np.einsum("n,n,na,nb->ab", amp, B, wh, wh))


@pytest.fixture(scope="module")
def corr_samples():
    prof = synthetic_rans_profile(180.0, 48)
    n_seeds = 8000
    ref = O.Sim(3, CORR_NY, 1, profile=prof, n_modes=100, t_filter=0.0, seed=0)
    tab, sc = ref.tables(), ref.scalars()
    Linv = []
    for j in range(CORR_NY):
        a6 = tab["a6"][j]
        Linv.append(np.linalg.inv(np.array([[a6[0], 0, 0], [a6[1], a6[2], 0], [a6[3], a6[4], a6[5]]])))
    prods = np.zeros((len(CORR_CASES), n_seeds, 3, 3))
    for s in range(n_seeds):
        sim = O.Sim(3, CORR_NY, 1, profile=prof, n_modes=100, t_filter=0.0, seed=s)
        for m, (j1, j2, dz, tau) in enumerate(CORR_CASES):
            # v' = a^-1 u' (eq. v_fluc) at two nodes and two times
            v1 = Linv[j1] @ sim.stg_raw(CORR_T0, j1, CORR_Z0)
            v2 = Linv[j2] @ sim.stg_raw(CORR_T0 + tau, j2, CORR_Z0 + dz)
            prods[m, s] = np.outer(v1, v2)
    # bulk velocity in lattice units from the unit scales (eq. u_transfer)
    U_b = prof.U_bulk * sc["c_t"] / sc["c_x"]
    c0 = 2.0 * math.pi * U_b / tab["l_e"].max()
    return prods, tab, c0


def _check_case(prods, tab, c0, m):
    j1, j2, dz, tau = CORR_CASES[m]
    p = prods[m]
    n = p.shape[0]
    mean = p.mean(0)
    se = p.std(0) / math.sqrt(n)
    cf = _corr_closed_form(tab["q"][j1], tab["q"][j2], tab["kn"], c0, j2 - j1, dz, tau)
    return mean, se, cf


def test_stg_time_correlation_closed_form(corr_samples):
    """At one node, trace <v'(t) . v'(t + tau)> = 3 sin(a)/a with a = c0 tau,
    and the tensor is diag(X, Y, Y) with X = 3 (sin a - a cos a)/a^3."""
    prods, tab, c0 = corr_samples
    for m, (j1, j2, dz, tau) in enumerate(CORR_CASES):
        if j1 != j2 or dz != 0:
            continue
        mean, se, cf = _check_case(prods, tab, c0, m)
        a = c0 * tau
        trace = 3.0 if a == 0 else 3.0 * math.sin(a) / a
        X = 1.0 if a == 0 else 3.0 * (math.sin(a) - a * math.cos(a)) / a ** 3
        np.testing.assert_allclose(np.trace(cf), trace, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(cf[0, 0], X, rtol=1e-9, atol=1e-12)
        tr_se = math.sqrt(float(np.sum(se.diagonal() ** 2)))
        assert abs(np.trace(mean) - trace) < 4.5 * tr_se, (tau, np.trace(mean), trace, tr_se)
        assert np.all(np.abs(mean - cf) < 4.5 * se), (tau, mean, cf, se)


def test_stg_space_time_correlation_closed_form(corr_samples):
    """Two-point, two-time correlation tensor of v' over seeds against the
    closed form, entry by entry (the streamwise-spanwise and streamwise-
    wall-normal entries change sign if the pseudo-position advects the wrong
    way)."""
    prods, tab, c0 = corr_samples
    odd_seen = 0
    for m, (j1, j2, dz, tau) in enumerate(CORR_CASES):
        mean, se, cf = _check_case(prods, tab, c0, m)
        assert np.all(np.abs(mean - cf) < 4.5 * se), (CORR_CASES[m], mean, cf, se)
        # entries odd in U_b that the sample resolves by more than 10 standard errors
        for (a, b) in ((0, 2), (2, 0), (0, 1), (1, 0)):
            if abs(cf[a, b]) > 10 * se[a, b]:
                odd_seen += 1
    assert odd_seen >= 4
