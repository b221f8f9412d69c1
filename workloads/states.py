"""Seeded population fields for starting two implementations from one state.

A field is 19 positive arrays f[i][z][y][x] (population-major, x fastest) of
the form  f_i = w_i (1 + a * smooth_i + b * white_i),  where smooth_i is a
sum of a few random low-wavenumber cosines (so the field has a smooth
density/velocity content plus a small cell-to-cell part) and w_i is the usual
D3Q19 weight of population i, used only as a scale.  Any positive field is a
valid starting state; no step of the method is evaluated here.

``D3Q19_ORDER`` is the velocity order of the 19 populations that the C-ABI
documents for every population array it exchanges.
"""
from __future__ import annotations

import numpy as np

D3Q19_ORDER = np.array([
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
    (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
    (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
], dtype=np.int64)

_W_SCALE = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _smooth(rng, nx, ny, nz, modes=3):
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    out = np.zeros((nz, ny, nx))
    for _ in range(modes):
        kx, ky, kz = rng.integers(0, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        out = out + rng.normal() * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
    return out / np.sqrt(modes)


def perturbed_equilibrium_field(nx, ny, nz, seed=0, smooth_amp=0.1,
                                white_amp=2e-3, dtype=np.float64):
    """Positive population field f[19][nz][ny][nx] around the rest weights."""
    rng = np.random.default_rng(seed)
    f = np.empty((19, nz, ny, nx))
    for i in range(19):
        s = _smooth(rng, nx, ny, nz)
        wn = rng.standard_normal((nz, ny, nx))
        f[i] = _W_SCALE[i] * (1.0 + smooth_amp * s + white_amp * wn)
    return np.ascontiguousarray(f.astype(dtype))
