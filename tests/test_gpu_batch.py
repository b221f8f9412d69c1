"""Batch executor and serving loop (GPU, through the C ABI).

A member of a batch runs exactly the kernels it runs alone, so every result
must be bit-identical alone and in the mix, whatever the members' sizes,
storages, boundary conditions, sampling periods and step phases; the serving
loop must return, for every job, the result of the same job run alone."""
import numpy as np
import pytest

from workloads import case
from workloads.serving import Job, channel_case

from gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu

SMALL = case("channel_64x32x32")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def _cases():
    return [
        SMALL.with_(nx=64, ny=16, nz=12, stats_every=5, seed=3),
        SMALL.with_(nx=96, ny=12, nz=18, stats_every=10, storage="fp16s", seed=4),
        SMALL.with_(nx=40, ny=10, nz=8, stats_every=0, bc_x="periodic", collision="bgk", force=(2e-6, 0.0, 1e-6)),
        SMALL.with_(nx=37, ny=9, nz=7, stats_every=2, seed=5),  # odd nx: scalar kernels
    ]


def _alone(c, steps):
    from paper_2205_02774_gb300.channel import Channel
    g = Channel.from_case(c, check_every=6, mass_tol=0.5)
    g.step(steps)
    st = g.stats()
    f = g.get_state()
    g.close()
    return f, st


def _same(f, st, ref):
    assert st["rc"] == 0, st["error"]
    assert np.array_equal(f, ref[0])
    assert np.array_equal(st["mean_sum"], ref[1]["mean_sum"])
    assert np.array_equal(st["rey_sum"], ref[1]["rey_sum"])
    assert st["n_samples"] == ref[1]["n_samples"]
    assert st["step"] == ref[1]["step"]


def test_batch_bit_identical_to_alone():
    from paper_2205_02774_gb300.channel import Channel
    from paper_2205_02774_gb300.serving import Batch
    cs = _cases()
    total = 40
    refs = [_alone(c, total) for c in cs]
    chans = [Channel.from_case(c, check_every=6, mass_tol=0.5) for c in cs]
    pre = [3, 0, 7, 1]  # different step phases when joining
    for ch, k in zip(chans, pre):
        ch.step(k)
    b = Batch()
    for ch in chans:
        b.add(ch)
    assert len(b) == len(cs)
    assert b.block_steps % 10 == 0 and b.block_steps >= 16
    b.step(30)  # one block and a remainder
    b.remove(chans[0])
    b.step(2)
    for ch, k in zip(chans, pre):
        done = k + 30 + (2 if ch is not chans[0] else 0)
        if ch in b.members:
            b.remove(ch)
        ch.step(total - done)
    for ch, ref in zip(chans, refs):
        _same(ch.get_state(), ch.stats(), ref)
        ch.close()
    b.close()


def test_batch_autotune_and_member_rules():
    from paper_2205_02774_gb300.capi import StgError
    from paper_2205_02774_gb300.channel import Channel
    from paper_2205_02774_gb300.serving import Batch
    cs = _cases()[:2]
    refs = [_alone(c, 124) for c in cs]
    chans = [Channel.from_case(c, check_every=6, mass_tol=0.5) for c in cs]
    b = Batch()
    for ch in chans:
        b.add(ch)
    b.step(4)
    tile = b.autotune(2)
    assert tile[0] in (0, 1)
    for ch in chans:
        assert ch.tile() == tile
        with pytest.raises(StgError):
            ch.step(1)
        with pytest.raises(StgError):
            ch.set_tile(1, 8, 24)
        with pytest.raises(StgError):
            ch.set_state(ch.get_state(), 0)
    b.step(120)  # the first blocks after a change run the members' own graphs, later ones the combined graph
    for ch, ref in zip(chans, refs):
        _same(ch.get_state(), ch.stats(), ref)
    chans[1].close()  # destroying a member takes it out of the batch
    assert len(b) == 1
    b.close()
    chans[0].step(1)  # usable alone after the batch is gone
    chans[0].close()


def _jobs():
    # arrivals close together and a few hundred steps each, so the jobs overlap
    specs = [(0.000, 4, 180, "fp32", 400), (0.001, 5, 395, "fp16s", 333), (0.002, 4, 395, "fp32", 250),
             (0.003, 6, 180, "fp32", 500), (0.004, 5, 180, "fp16s", 210), (0.050, 4, 180, "fp32", 300)]
    return [Job(t, channel_case(h, re, st, seed=i + 1, n_modes=40, n_fv=48), steps)
            for i, (t, h, re, st, steps) in enumerate(specs)]


def test_serve_results_equal_alone():
    from paper_2205_02774_gb300.serving import serve
    jobs = _jobs()
    results, rep = serve(jobs, hbm_budget_bytes=8e9, check_every=6, keep_stats=True)
    assert rep["completed"] == len(jobs) and rep["failed"] == 0
    assert rep["peak_active"] >= 2  # the jobs overlapped
    assert rep["p99_latency_s"] >= rep["p50_latency_s"] > 0
    assert rep["cell_updates"] == sum(j.case.cells * j.steps for j in jobs)
    for jb, r in zip(jobs, results):
        assert r["status"] == 0
        assert r["admit_s"] >= jb.arrival_s - 1e-9
        assert r["finish_s"] >= r["admit_s"]
        _, st = _alone(jb.case, jb.steps)
        assert np.array_equal(r["mean_sum"], st["mean_sum"])
        assert np.array_equal(r["rey_sum"], st["rey_sum"])
        assert r["n_samples"] == st["n_samples"]


def test_serve_memory_budget():
    from paper_2205_02774_gb300 import capi as A
    from paper_2205_02774_gb300.channel import case_kwargs, create_structs
    from paper_2205_02774_gb300.serving import serve
    # four jobs of one size: the budget holds exactly one of them
    jobs = [Job(0.001 * i, channel_case(5, 180, "fp32", seed=20 + i, n_modes=40, n_fv=48), 120) for i in range(4)]
    est = []
    for jb in jobs:
        c = jb.case
        d, _, p, _ = create_structs(c.nx, c.ny, c.nz, **case_kwargs(c))
        est.append(A.stg_lbm_estimate_bytes(d, p))
    budget = max(est) * 1.01  # room for one job at a time
    big = Job(0.0, channel_case(12, 180, "fp32", seed=9, n_modes=40, n_fv=48), 5)  # larger than the budget
    results, rep = serve(jobs + [big], hbm_budget_bytes=budget, check_every=6)
    assert rep["peak_active"] == 1
    assert [r["status"] for r in results[:4]] == [0, 0, 0, 0]
    assert results[4]["status"] == A.STG_ERR_NOMEM
    assert rep["completed"] == 4 and rep["failed"] == 1


@pytest.mark.parametrize("kw", [dict(), dict(storage="fp16s"), dict(stats_every=0), dict(bc_x="periodic"),
                                dict(sponge_len=10.0), dict(n_modes=0)])
def test_admission_estimate_bounds_the_allocation(kw):
    """The serving loop admits jobs by stg_lbm_estimate_bytes; it must not
    undercount what create() really allocates."""
    from paper_2205_02774_gb300 import capi as A
    from paper_2205_02774_gb300.channel import Channel, case_kwargs, create_structs
    c = SMALL.with_(nx=96, ny=20, nz=18, **kw)
    d, _, p, _ = create_structs(c.nx, c.ny, c.nz, **case_kwargs(c))
    est = A.stg_lbm_estimate_bytes(d, p)
    g = Channel.from_case(c)
    used = g.info()["device_bytes"]
    g.close()
    assert used <= est <= 1.5 * used + 4e6


def _oracle_200():
    import oracle as O
    c = SMALL  # 64x32x32, 100 modes, statistics every 10 steps
    o = O.Sim.from_case(c)
    o.step(200)
    m, r, n = o.stats()
    return o.pops(), m, r, n


def _fluct(mean_sum, rey_sum, n, nz):
    cnt = n * nz
    return rey_sum[0] / cnt - (mean_sum[0] / cnt) ** 2


def test_batch_and_served_members_match_oracle():
    """Batched and served forms against the FP64 oracle: the 64x32x32 channel
    run for 200 steps as a member of a batch (beside members of other sizes and
    an FP16 copy of itself) and as a job of the serving loop (beside other
    jobs) gives the oracle's velocity and statistics, FP32 storage at 1e-4
    normwise (the single-channel parity bound), FP16 storage at 1e-2."""
    from paper_2205_02774_gb300.channel import Channel
    from paper_2205_02774_gb300.serving import Batch, serve
    from gpu_helpers import velocity, normwise
    fo, mo, ro, no = _oracle_200()
    c = SMALL
    chans = [Channel.from_case(c, check_every=20, mass_tol=0.1),
             Channel.from_case(c.with_(storage="fp16s"), check_every=20, mass_tol=0.1),
             Channel.from_case(_cases()[0], check_every=6, mass_tol=0.5),
             Channel.from_case(_cases()[1], check_every=6, mass_tol=0.5)]
    b = Batch()
    for ch in chans:
        b.add(ch)
    b.step(200)
    errs = {}
    for name, ch, tol in (("fp32", chans[0], 1e-4), ("fp16s", chans[1], 1e-2)):
        st = ch.stats()
        assert st["rc"] == 0, st["error"]
        assert st["n_samples"] == no == 20
        errs[name] = (normwise(velocity(ch.populations()), velocity(fo)), normwise(st["mean_sum"], mo),
                      normwise(st["rey_sum"], ro),
                      normwise(_fluct(st["mean_sum"], st["rey_sum"], no, c.nz), _fluct(mo, ro, no, c.nz)))
        assert max(errs[name][:3]) < tol, (name, errs[name])
        assert errs[name][3] < (1e-2 if name == "fp32" else 5e-2), (name, errs[name])
    b.close()
    for ch in chans:
        ch.close()
    # the same channel as a served job among others arriving at the same time
    jobs = [Job(0.0, SMALL, 200)] + _jobs()[:3]
    results, rep = serve(jobs, hbm_budget_bytes=8e9, check_every=20, keep_stats=True)
    assert rep["completed"] == len(jobs)
    r0 = results[0]
    assert r0["status"] == 0 and r0["n_samples"] == no
    errs["served"] = (normwise(r0["mean_sum"], mo), normwise(r0["rey_sum"], ro))
    assert max(errs["served"]) < 1e-4, errs
    print("batched / served vs oracle", errs)
