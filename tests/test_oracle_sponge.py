"""Pins of the oracle's sponge zone, eq. (sponge_visco) of Sec. IV:
nu_sponge = nu_eff [K ((x - x_start)/(x_end - x_start))^p + 1].

* the factor at the zone's start, middle and end, and 1 before the zone;
* K = 0 reproduces the run without a sponge exactly;
* a Taylor-Green vortex inside a zone of constant factor (p = 0 over the
  whole domain) decays at the analytic rate of the scaled viscosity
  F nu = F c_s^2 (tau - 1/2), which fixes how the factor enters the
  relaxation time."""
import math

import numpy as np
import pytest

import oracle as O
from workloads import perturbed_equilibrium_field

from test_oracle_flows import velocity_of_stored


def test_sponge_factor_closed_form():
    d = O.make_domain(101, 4, 4, sponge=(40.0, 1000.0, 3.0))  # x_end = 100, x_start = 60
    assert O.sponge_factor(d, 0) == 1.0
    assert O.sponge_factor(d, 59) == 1.0
    assert O.sponge_factor(d, 60) == 1.0
    assert O.sponge_factor(d, 80) == pytest.approx(1.0 + 1000.0 * 0.5 ** 3, rel=1e-15)  # 126
    assert O.sponge_factor(d, 90) == pytest.approx(1.0 + 1000.0 * 0.75 ** 3, rel=1e-15)
    assert O.sponge_factor(d, 100) == pytest.approx(1001.0, rel=1e-15)
    vals = [O.sponge_factor(d, x) for x in range(60, 101)]
    assert all(b > a for a, b in zip(vals, vals[1:]))
    off = O.make_domain(101, 4, 4, sponge=(0.0, 1000.0, 3.0))
    assert all(O.sponge_factor(off, x) == 1.0 for x in range(101))


def test_sponge_with_zero_K_is_no_sponge():
    f = perturbed_equilibrium_field(24, 6, 5, seed=8)
    a = O.Sim(24, 6, 5, bc_x="periodic", bc_y="walls", force=(1e-5, 0.0, 0.0))
    b = O.Sim(24, 6, 5, bc_x="periodic", bc_y="walls", force=(1e-5, 0.0, 0.0), sponge=(10.0, 0.0, 3.0))
    c = O.Sim(24, 6, 5, bc_x="periodic", bc_y="walls", force=(1e-5, 0.0, 0.0), sponge=(10.0, 1000.0, 3.0))
    for s in (a, b, c):
        s.set_pops(f)
        s.step(3)
    assert np.array_equal(a.pops(), b.pops())
    diff = np.abs(c.pops() - a.pops()).max(axis=(0, 1, 2))  # per x column
    # the zone starts at x = 13 (factor 1 there); in 3 steps its effect reaches
    # 3 columns to each side, across the periodic x wrap too
    assert diff[3:11].max() == 0.0
    assert diff[14:].min() > 0.0


@pytest.mark.parametrize("collision", ["regularized", "bgk"])
@pytest.mark.parametrize("K", [1.0, 3.0])
def test_taylor_green_decay_in_constant_sponge(collision, K):
    N = 32
    tau = 0.56
    nu = (1.0 + K) * (tau - 0.5) / 3.0
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
    # p = 0 with the zone covering x = 0 .. N-1: factor 1 + K everywhere
    s = O.Sim(N, N, 1, tau0=tau, c_smag=0.0, bc_x="periodic", bc_y="periodic", collision=collision,
              sponge=(float(N - 1), K, 0.0))
    assert all(O.sponge_factor(s.domain, xx) == 1.0 + K for xx in range(N))
    s.set_pops(f)

    def energy():
        u = velocity_of_stored(s.pops())
        return float((u ** 2).sum())

    s.step(20)
    e1 = energy()
    s.step(100)
    e2 = energy()
    rate = -math.log(e2 / e1) / 100
    assert rate == pytest.approx(4 * nu * k * k, rel=1e-2)
