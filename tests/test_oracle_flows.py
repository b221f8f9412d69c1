"""Whole-step pins of the oracle: exact discrete Poiseuille solutions, the
Taylor-Green viscous decay rate, mass conservation, a uniform plug flow
through inlet and outlet, and a brute-force transcription on a 4x4x4 lattice."""
import math

import numpy as np
import pytest

import oracle as O
from workloads import RansProfile, perturbed_equilibrium_field, D3Q19_ORDER, case

from bruteforce_lbm import step as bf_step

C3 = D3Q19_ORDER.astype(np.float64)


def velocity_of_stored(f, F=(0.0, 0.0, 0.0)):
    """Velocity of a stored (post-collision) lattice: the stored momentum
    already holds the full force of the step, so u = (sum c f - F/2)/rho."""
    rho = f.sum(0)
    j = np.einsum("ia,i...->a...", C3, f)
    return (j - 0.5 * np.asarray(F).reshape(3, *([1] * (f.ndim - 1)))) / rho


@pytest.mark.parametrize("collision,lam", [("bgk", lambda t: (t - 0.5) ** 2),
                                           ("regularized", lambda t: (t - 0.5) * 0.5)])
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_poiseuille_exact_discrete_solution(collision, lam, tau):
    """Half-way bounce-back Poiseuille flow: the steady lattice solution is the
    parabola F/(2 nu) y (H - y) plus a uniform slip F/(2 nu) (16 L - 3)/12,
    with L = (tau+ - 1/2)(tau- - 1/2) the two-relaxation-time 'magic'
    product (Ginzburg & d'Humieres).  BGK has tau- = tau; the regularized
    collision resets the odd non-hydrodynamic moments, i.e. tau- = 1."""
    ny, F = 32, 1e-6
    nu = (tau - 0.5) / 3
    s = O.Sim(1, ny, 1, tau0=tau, c_smag=0.0, force=(F, 0, 0), bc_x="periodic", bc_y="walls",
              collision=collision)
    s.step(int(8 * ny * ny / nu))
    ux = velocity_of_stored(s.pops(), (F, 0, 0))[0, 0, :, 0]
    y = np.arange(ny) + 0.5
    L = lam(tau)
    exact = F / (2 * nu) * (y * (ny - y) + (16 * L - 3) / 12)
    np.testing.assert_allclose(ux, exact, rtol=0, atol=1e-7 * exact.max())
    # and the textbook parabola within the O(1/H^2) wall-closure error
    para = F / (2 * nu) * y * (ny - y)
    assert np.abs(ux - para).max() / para.max() < 1e-3


@pytest.mark.parametrize("collision", ["regularized", "bgk"])
@pytest.mark.parametrize("tau", [0.6, 0.8])
def test_taylor_green_decay_rate(collision, tau):
    N = 32
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / N
    u0 = 0.01
    x = np.arange(N)[None, :]
    y = np.arange(N)[:, None]
    ux = -u0 * np.cos(k * x) * np.sin(k * y)
    uy = u0 * np.sin(k * x) * np.cos(k * y)
    f = np.zeros((19, 1, N, N))
    for yy in range(N):
        for xx in range(N):
            f[:, 0, yy, xx] = O.equilibrium(1.0, [ux[yy, xx], uy[yy, xx], 0.0])
    s = O.Sim(N, N, 1, tau0=tau, c_smag=0.0, bc_x="periodic", bc_y="periodic", collision=collision)
    s.set_pops(f)

    def energy():
        u = velocity_of_stored(s.pops())
        return float((u ** 2).sum())

    s.step(20)
    e1 = energy()
    s.step(200)
    e2 = energy()
    rate = -math.log(e2 / e1) / 200
    assert rate == pytest.approx(4 * nu * k * k, rel=1e-2)


def test_mass_conservation_periodic_box():
    n = 8
    f = perturbed_equilibrium_field(n, n, n, seed=3)
    s = O.Sim(n, n, n, tau0=0.52, c_smag=0.01, bc_x="periodic", bc_y="periodic")
    s.set_pops(f)
    m0 = f.sum()
    s.step(1000)
    assert abs(s.pops().sum() - m0) / m0 < 1e-13
    assert abs(s.mass - m0) / m0 < 1e-13


def _plug_profile(U):
    n = 48
    from workloads import tanh_grid
    faces = tanh_grid(n)
    y_c = 0.5 * (faces[1:] + faces[:-1])
    return RansProfile(y_c=y_c, U=np.full(n, U), k=np.zeros(n), eps=np.ones(n), R=np.zeros((n, 6)),
                       U_bulk=U, nu_phys=1 / 180, h_phys=1.0, re_tau=180.0)


def test_uniform_plug_flow_through_inlet_and_outlet():
    """No fluctuations (R = 0, k = 0) and a uniform RANS velocity with periodic
    y: the whole lattice is a fixed point of inlet, outlet and collision."""
    nx, ny, nz = 12, 16, 4
    prof = _plug_profile(10.0)
    s = O.Sim(nx, ny, nz, tau0=0.55, c_smag=0.01, bc_x="stg", bc_y="periodic", profile=prof,
              n_modes=16, t_filter=3.0, mach_target=0.05)
    f0 = s.pops()
    u_lb = s.scalars()["U_b"]
    assert u_lb == pytest.approx(0.05 * math.sqrt(1 / 3), rel=1e-14)
    np.testing.assert_allclose(f0[:, 0, 0, 0], O.equilibrium(1.0, [u_lb, 0, 0]), atol=1e-16)
    s.step(50)
    np.testing.assert_allclose(s.pops(), f0, atol=2e-15)
    np.testing.assert_allclose(s.inlet()[0], u_lb, rtol=1e-14)


@pytest.mark.parametrize("collision", ["regularized", "bgk"])
def test_bruteforce_4x4x4_all_boundaries(collision):
    c = case("channel_64x32x32").with_(nx=4, ny=4, nz=4, n_modes=20, collision=collision,
                                       stats_every=0, t_filter=2.0)
    s = O.Sim.from_case(c)
    f = perturbed_equilibrium_field(4, 4, 4, seed=11)
    s.set_pops(f)
    ref = f.copy()
    for _ in range(10):
        s.step(1)
        ub = s.inlet()
        ref = np.array(bf_step(ref, (4, 4, 4), D3Q19_ORDER, c.tau0, c.c_smag, c.force, ub,
                               regularized=(collision == "regularized")))
        np.testing.assert_allclose(s.pops(), ref, rtol=1e-13, atol=0)


def test_bruteforce_periodic_force():
    f = perturbed_equilibrium_field(4, 3, 5, seed=5)
    F = (2e-4, -1e-4, 3e-5)
    s = O.Sim(4, 3, 5, tau0=0.57, c_smag=0.02, force=F, bc_x="periodic", bc_y="walls")
    s.set_pops(f)
    ref = f.copy()
    for _ in range(5):
        s.step(1)
        ref = np.array(bf_step(ref, (4, 3, 5), D3Q19_ORDER, 0.57, 0.02, F, None, bc_x="periodic"))
    np.testing.assert_allclose(s.pops(), ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("every,chunks", [(5, (50,)), (5, (7, 5, 38)), (3, (1, 1, 20)), (1, (4,))])
def test_plug_flow_statistics_accumulation(every, chunks):
    """Running statistics (eqs. y_plus, v_rms: time- and span-averaged u and
    u u): in the uniform plug flow every sampled step adds nz U to sum u_x and
    nz U^2 to sum u_x u_x of each (x, y), nothing to the other sums, and a
    sample is taken after step t exactly when (t + 1) is a multiple of the
    sampling period, however the steps are split into calls."""
    nx, ny, nz = 12, 16, 4
    prof = _plug_profile(10.0)
    s = O.Sim(nx, ny, nz, tau0=0.55, c_smag=0.01, bc_x="stg", bc_y="periodic", profile=prof,
              n_modes=16, t_filter=3.0, mach_target=0.05, stats_every=every)
    U = s.scalars()["U_b"]
    total = 0
    for k in chunks:
        s.step(k)
        total += k
        m, r, n = s.stats()
        assert n == total // every
        np.testing.assert_allclose(m[0], n * nz * U, rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(m[1:], 0.0, atol=1e-15 * nz * max(n, 1))
        np.testing.assert_allclose(r[0], n * nz * U * U, rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(r[1:], 0.0, atol=1e-15 * nz * max(n, 1))
