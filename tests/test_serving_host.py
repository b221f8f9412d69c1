"""Host-side pieces of the batched and served workloads (no GPU): the job
stream recipes and the admission estimate of the C library (a pure host
computation)."""
import numpy as np
import pytest

from workloads.serving import ensemble, poisson_stream


def test_poisson_stream_recipe():
    jobs = poisson_stream(500, rate_per_s=2.0, seed=7)
    assert len(jobs) == 500
    t = np.array([j.arrival_s for j in jobs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(0.5, rel=0.1)  # mean inter-arrival 1/rate
    for j in jobs:
        h = j.case.ny // 2
        assert (j.case.nx, j.case.ny, j.case.nz) == (12 * h, 2 * h, 3 * h)
        assert 0.5e6 <= j.case.cells <= 20e6
        assert 1000 <= j.steps <= 20000
        assert j.case.storage in ("fp32", "fp16sr") and j.case.re_tau in (180.0, 395.0)
    assert [j.case.seed for j in jobs] == list(range(500))
    again = poisson_stream(500, rate_per_s=2.0, seed=7)
    assert [(j.arrival_s, j.case, j.steps) for j in jobs] == [(j.arrival_s, j.case, j.steps) for j in again]


def test_ensemble_recipe():
    jobs = ensemble(64)
    assert len(jobs) == 64 and all(j.arrival_s == 0.0 and j.steps == 5000 for j in jobs)
    assert {j.case.ny // 2 for j in jobs} <= {16, 24, 32, 48, 64}
    assert [j.case.seed for j in jobs] == list(range(1, 65))


def test_estimate_bytes_bounds():
    from paper_2205_02774_gb300 import capi as A
    from paper_2205_02774_gb300.channel import case_kwargs, create_structs
    from workloads.serving import channel_case
    prev = 0
    for h in (8, 16, 32):
        for storage, elem in (("fp32", 4), ("fp16s", 2)):
            c = channel_case(h, 180, storage)
            d, _, p, _ = create_structs(c.nx, c.ny, c.nz, **case_kwargs(c))
            est = A.stg_lbm_estimate_bytes(d, p)
            lattices = 2 * 19 * c.cells * elem
            assert lattices <= est <= lattices * 1.2 + 8e6
        assert est > prev
        prev = est
