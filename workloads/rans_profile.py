"""Closed-form stand-in for the RANS interface profile of a plane channel.

The paper feeds its synthetic turbulence generator from a k-omega RANS solve of
a Re_tau = 180 channel on a 96-cell wall-normal finite-volume grid whose cells
grow towards the centre (Sec. IV). That solver is outside this project, so the
profile is synthesised here from closed forms in wall units (u_tau = 1,
nu = 1/Re_tau, half-height h = 1 m):

* mean velocity: Reichardt's law of the wall, mirrored about the centreline;
* turbulent kinetic energy  k+ = 18 s/(1+s)^2 + 0.8 (1 - exp(-y+/30)),
  s = (y+/15)^2  (near-wall peak of about 4.8 at y+ = 15, about 0.9 at the centre);
* dissipation  eps+ = 1 / (kappa (y+ + 8));
* Reynolds stresses  R11 = 1.1 k, R22 = 0.4 k, R33 = 0.5 k (trace 2k),
  R12 = -(1 - y/h)(1 - exp(-y+/26))^2 (antisymmetric about the centreline),
  R13 = R23 = 0.

Values are given at the cell centres of a tanh-stretched grid
y_i = h [1 + tanh(beta (2 i/n - 1)) / tanh(beta)], i = 0..n.

These are inputs, not part of the method: the same arrays are handed to the
CUDA library and to the CPU oracle.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

KAPPA = 0.41


def tanh_grid(n_cells: int, beta: float = 2.0, h: float = 1.0) -> np.ndarray:
    """Face coordinates (n_cells + 1) of a tanh-stretched grid over [0, 2h]."""
    i = np.arange(n_cells + 1, dtype=np.float64)
    return h * (1.0 + np.tanh(beta * (2.0 * i / n_cells - 1.0)) / np.tanh(beta))


@dataclass
class RansProfile:
    """A 1-D wall-normal RANS profile on finite-volume cell centres.

    ``R`` is (n, 6) with columns 11, 22, 33, 12, 13, 23.  All arrays are float64,
    physical units (m, m/s, m^2/s^2, m^2/s^3).
    """

    y_c: np.ndarray
    U: np.ndarray
    k: np.ndarray
    eps: np.ndarray
    R: np.ndarray
    U_bulk: float
    nu_phys: float
    h_phys: float
    re_tau: float

    @property
    def n_fv(self) -> int:
        return int(self.y_c.shape[0])

    @property
    def U_max(self) -> float:
        return float(self.U.max())


def reichardt_u_plus(y_plus: np.ndarray) -> np.ndarray:
    yp = np.asarray(y_plus, dtype=np.float64)
    return (np.log1p(KAPPA * yp) / KAPPA
            + 7.8 * (1.0 - np.exp(-yp / 11.0) - (yp / 11.0) * np.exp(-yp / 3.0)))


def synthetic_rans_profile(re_tau: float = 180.0, n_cells: int = 48,
                           beta: float = 2.0) -> RansProfile:
    """Synthetic channel profile in wall units (u_tau = 1, h = 1, nu = 1/Re_tau)."""
    h = 1.0
    nu = 1.0 / re_tau
    faces = tanh_grid(n_cells, beta, h)
    y_c = 0.5 * (faces[:-1] + faces[1:])
    dy = np.diff(faces)
    y_wall = np.minimum(y_c, 2.0 * h - y_c)
    yp = y_wall / nu
    U = reichardt_u_plus(yp)
    s = (yp / 15.0) ** 2
    k = 18.0 * s / (1.0 + s) ** 2 + 0.8 * (1.0 - np.exp(-yp / 30.0))
    eps_plus = 1.0 / (KAPPA * (yp + 8.0))
    eps = eps_plus / nu  # eps = eps+ u_tau^4 / nu
    R = np.zeros((n_cells, 6))
    R[:, 0] = 1.1 * k
    R[:, 1] = 0.4 * k
    R[:, 2] = 0.5 * k
    R[:, 3] = -(1.0 - y_c / h) * (1.0 - np.exp(-yp / 26.0)) ** 2
    U_bulk = float(np.sum(U * dy) / (2.0 * h))
    return RansProfile(y_c=y_c, U=U, k=k, eps=eps, R=R, U_bulk=U_bulk,
                       nu_phys=nu, h_phys=h, re_tau=float(re_tau))
