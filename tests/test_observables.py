"""Post-processing of Sec. V (host logic) against closed forms.

* mean and Reynolds stress from sums of known samples;
* eq. (u_shear) on the exact laminar Poiseuille profile: the first-order wall
  gradient gives u_tau^2 = F (h - 1/4), i.e. u_tau / sqrt(F h) =
  sqrt(1 - 1/(4h)) (force balance u_theory = sqrt(F h));
* wall units of a linear profile;
* B_uu of a pure cosine and eq. (time-integral) of a known B."""
import math

import numpy as np
import pytest

from paper_2205_02774_gb300 import observables as ob


def test_mean_and_stress_from_sums():
    rng = np.random.default_rng(0)
    ny, nx, nz, n = 4, 5, 3, 7
    u = rng.normal(size=(n, nz, 3, ny, nx))  # samples over steps and z
    ms = u.sum(axis=(0, 1))
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    rs = np.stack([(u[:, :, a] * u[:, :, b]).sum(axis=(0, 1)) for a, b in pairs])
    U, R = ob.mean_and_stress(ms, rs, n, nz)
    flat = u.reshape(n * nz, 3, ny, nx)
    np.testing.assert_allclose(U, flat.mean(0), rtol=1e-13)
    for k, (a, b) in enumerate(pairs):
        ref = ((flat[:, a] - flat[:, a].mean(0)) * (flat[:, b] - flat[:, b].mean(0))).mean(0)
        np.testing.assert_allclose(R[k], ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("h", [8, 32, 90])
def test_friction_velocity_poiseuille(h):
    F, nu = 1e-6, 0.02
    ny = 2 * h
    y = np.arange(ny) + 0.5
    Ux = F / (2 * nu) * y * (ny - y)
    ut = ob.friction_velocity(Ux, nu)
    assert ut == pytest.approx(math.sqrt(F * (h - 0.25)), rel=1e-13)
    assert ut / ob.u_theory_force(F, h) == pytest.approx(math.sqrt(1 - 1 / (4 * h)), rel=1e-13)


def test_wall_units_linear_profile():
    ny, nx, nu = 20, 3, 0.01
    y = np.arange(ny) + 0.5
    g = 0.004
    U = np.zeros((3, ny, nx))
    U[0] = (g * np.minimum(y, ny - y))[:, None]
    R = np.zeros((6, ny, nx))
    R[0] = 4e-6
    yp, up, rms, ut = ob.wall_units(U, R, nu, 1, half="both")
    assert ut == pytest.approx(math.sqrt(nu * g), rel=1e-13)
    np.testing.assert_allclose(yp, y[:10] * ut / nu, rtol=1e-13)
    np.testing.assert_allclose(up, g * y[:10] / ut, rtol=1e-13)  # u+ = y+ in a linear (viscous) layer
    np.testing.assert_allclose(rms[0], 2e-3 / ut, rtol=1e-13)
    assert ob.u_theory_re(180.0, nu, ny / 2) == pytest.approx(180 * nu / 10)


def test_autocorrelation_of_cosine_and_integral_time():
    P = 64
    t = np.arange(P * 200)
    B = ob.autocorrelation(np.cos(2 * np.pi * t / P), max_lag=P)
    np.testing.assert_allclose(B, np.cos(2 * np.pi * np.arange(P + 1) / P), atol=2e-3)
    # eq. (time-integral) of B = cos(pi t / (2 t0)) up to its zero at t0: 2 t0 / pi
    t0, dt = 10.0, 0.001
    tt = np.arange(0, 2 * t0, dt)
    Bk = np.cos(np.pi * tt / (2 * t0))
    assert ob.integral_time(Bk, dt) == pytest.approx(2 * t0 / np.pi, rel=1e-6)
    # exponential never crosses zero: the whole record is integrated
    Be = np.exp(-tt / 3.0)
    assert ob.integral_time(Be, dt) == pytest.approx(3.0 * (1 - np.exp(-tt[-1] / 3.0)), rel=1e-6)
