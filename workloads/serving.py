"""Synthetic job streams for the batched and served channel workloads.

Every job is an STG channel of half-height h on a 12h x 2h x 3h lattice
(the production channel's aspect) with its own Re_tau, storage, step count
and seed.  Two recipes:

* ensemble(n, ...): n channels with h drawn from a set of half-heights and
  Re_tau from {180, 395}, seeds 1..n, all present at time 0 (the batched
  ensemble);
* poisson_stream(n, rate, ...): n jobs arriving as a Poisson process; h is
  uniform on the integers whose lattice has between min_cells and max_cells
  cells, steps uniform in [steps_min, steps_max], storage uniform on
  {fp32, fp16sr} (binary16 written by stochastic rounding), Re_tau uniform
  on {180, 395}, seed = job id.

Only random draws live here; no step of the method is evaluated.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .configs import ChannelCase


@dataclass(frozen=True)
class Job:
    arrival_s: float
    case: ChannelCase
    steps: int


def channel_case(h, re_tau=180.0, storage="fp32", seed=0, n_modes=200, n_fv=96, stats_every=10, streaming="pull"):
    return ChannelCase(f"channel_h{h}", 12 * h, 2 * h, 3 * h, n_modes=n_modes, n_fv=n_fv, re_tau=float(re_tau),
                       seed=int(seed), storage=storage, stats_every=stats_every, streaming=streaming)


def ensemble(n, heights=(16, 24, 32, 48, 64), re_taus=(180, 395), steps=5000, draw_seed=12345, storage="fp32",
             n_modes=200):
    rng = np.random.default_rng(draw_seed)
    jobs = []
    for i in range(n):
        h = int(rng.choice(heights))
        re = float(rng.choice(re_taus))
        jobs.append(Job(0.0, channel_case(h, re, storage, seed=i + 1, n_modes=n_modes), int(steps)))
    return jobs


def poisson_stream(n, rate_per_s=2.0, min_cells=0.5e6, max_cells=20e6, steps_min=1000, steps_max=20000,
                   storages=("fp32", "fp16sr"), re_taus=(180, 395), seed=7, n_modes=200, streaming="pull"):
    rng = np.random.default_rng(seed)
    hs = [h for h in range(2, 1024) if min_cells <= 72 * h ** 3 <= max_cells]
    if not hs:
        raise ValueError("no half-height gives a lattice in the cell range")
    t = 0.0
    jobs = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        h = int(rng.choice(hs))
        steps = int(rng.integers(steps_min, steps_max + 1))
        storage = str(rng.choice(storages))
        re = float(rng.choice(re_taus))
        jobs.append(Job(t, channel_case(h, re, storage, seed=i, n_modes=n_modes, streaming=streaming), steps))
    return jobs
