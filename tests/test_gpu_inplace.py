"""The one-lattice in-place (AA-pattern) update against the oracle and
against the two-lattice pull scheme, through the C ABI.

Steps of even index read slot opp(i) of cell x - c_i and write slot i of
cell x + c_i; steps of odd index read slot i and write slot opp(i) of the same
cell.  Every cell does the same arithmetic as in the pull scheme, so the
canonical state (f*_i of cell x, what get_state returns) and the statistics
must be bit-identical to the pull scheme's (the mass to rounding), step after step,
whatever the step parity, storage, boundary conditions or launch tile; and a
single step from an identical state must match the oracle at the pull
scheme's tolerance (1e-5) on both parities."""
import numpy as np
import pytest

from workloads import case, perturbed_equilibrium_field

from gpu_helpers import require_cuda, pair, velocity, max_rel, normwise, fp16_bits, fp16_decode, fp16_half_ulp

pytestmark = pytest.mark.gpu

SMALL = case("channel_64x32x32")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def _run(c, steps, tile=None, **kw):
    from paper_2205_02774_gb300.channel import Channel
    g = Channel.from_case(c, check_every=kw.pop("check_every", 7), mass_tol=0.5, **kw)
    if tile:
        g.set_tile(*tile)
    out = []
    for n in steps:
        g.step(n)
        st = g.stats()
        assert st["rc"] == 0, st["error"]
        out.append((g.get_state(), st))
    info = g.info()
    g.close()
    return out, info


def _same(a, b):
    for (fa, sa), (fb, sb) in zip(a, b):
        assert np.array_equal(fa, fb)
        assert np.array_equal(sa["mean_sum"], sb["mean_sum"])
        assert np.array_equal(sa["rey_sum"], sb["rey_sum"])
        assert sa["n_samples"] == sb["n_samples"] and sa["step"] == sb["step"]
        # the FP64 mass adds the same values grouped by memory cell, i.e. in another order
        assert abs(sa["mass"] - sb["mass"]) <= 1e-9 * abs(sb["mass"])


@pytest.mark.parametrize("dims,kw", [
    ((64, 32, 32), dict()),
    ((64, 32, 32), dict(storage="fp16s")),
    ((64, 32, 32), dict(storage="fp16sr")),
    ((70, 10, 9), dict(collision="bgk", stats_every=3)),                          # ragged x chunk
    ((130, 6, 5), dict(bc_x="periodic", force=(2e-5, 0.0, 1e-5))),                # periodic x, walls, force
    ((64, 8, 4), dict(bc_x="periodic", bc_y="periodic", collision="bgk", force=(1e-5, -2e-5, 0.0))),
    ((260, 6, 5), dict(storage="fp16s", stats_every=1)),                          # 2-byte x halo, sampling every step
    ((96, 12, 18), dict(sponge_len=10.0)),
    ((4, 3, 2), dict(n_modes=7)),                                                 # smallest in-place lattice
    ((136, 6, 5), dict(storage="fp16sr", bc_x="periodic")),                       # quads, shuffled x halo
    ((200, 6, 5), dict(storage="fp16s", stats_every=2)),                          # quads, ragged last chunk
    ((8, 4, 3), dict(storage="fp16s", n_modes=7)),                                # smallest quad lattice
])
def test_inplace_bit_identical_to_pull(dims, kw):
    nx, ny, nz = dims
    c = SMALL.with_(nx=nx, ny=ny, nz=nz, **kw)
    steps = (1, 1, 5, 12)  # both parities, single steps and graph blocks
    ref, info_p = _run(c, steps)
    got, info_a = _run(c.with_(streaming="aa"), steps)
    _same(got, ref)
    # one lattice instead of two
    lat = 19 * c.cells * (4 if c.storage == "fp32" else 2)
    assert info_p["device_bytes"] - info_a["device_bytes"] >= lat - 4096


@pytest.mark.parametrize("tile", [(0, 0, 0), (1, 4, 24), (0, 16, 4), (1, 8, 8)])
def test_inplace_tiles_bit_identical(tile):
    c = SMALL.with_(nx=256, ny=12, nz=20, streaming="aa", stats_every=5)
    ref, _ = _run(c, (3, 20), tile=(1, 8, 24))
    got, _ = _run(c, (3, 20), tile=tile)
    _same(got, ref)


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
@pytest.mark.parametrize("start", [0, 1])
def test_inplace_single_step_vs_oracle(storage, start):
    """One step from an identical state at an even (shifted) and an odd
    (local) step index, every population against the oracle.  The oracle is
    brought to the same step index first, so both use the inlet plane of that
    step (temporal filter off: set_state restarts it)."""
    c = SMALL.with_(nx=66, ny=10, nz=7, stats_every=0, storage=storage, streaming="aa", t_filter=0.0)
    gpu, orc = pair(c)
    orc.step(start)
    f = perturbed_equilibrium_field(c.nx, c.ny, c.nz, seed=5 + start)
    if storage == "fp32":
        st = gpu.encode(f)
        orc.set_pops(gpu.decode(st))
    else:
        st = fp16_bits(f)
        orc.set_pops(fp16_decode(st))
    gpu.set_state(st, start)
    assert np.array_equal(gpu.get_state(), st)  # the canonical round trip at this parity
    gpu.step(1)
    orc.step(1)
    fo = orc.pops()
    if storage == "fp32":
        assert max_rel(gpu.populations(), fo) < 1e-5
    else:
        W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12).reshape(19, 1, 1, 1)
        excess = np.abs(fp16_decode(gpu.get_state()) - fo) - (fp16_half_ulp(fo - W) + 2e-6 * np.abs(fo))
        assert excess.max() <= 0


def test_inplace_200_steps_channel_vs_oracle():
    c = SMALL.with_(streaming="aa")
    gpu, orc = pair(c, check_every=20, mass_tol=0.1)
    gpu.step(c.steps)
    orc.step(c.steps)
    fg, fo = gpu.populations(), orc.pops()
    assert normwise(velocity(fg), velocity(fo)) < 1e-4
    st = gpu.stats()
    m, r, n = orc.stats()
    assert st["rc"] == 0 and st["n_samples"] == n
    assert normwise(st["mean_sum"], m) < 1e-4 and normwise(st["rey_sum"], r) < 1e-4


@pytest.mark.parametrize("start", [0, 1])
def test_inplace_block_probes_checkpoint(start):
    """Sub-block read-back, probes and checkpoints of an in-place lattice at
    both step parities."""
    from paper_2205_02774_gb300.channel import Channel
    c = SMALL.with_(nx=64, ny=16, nz=12, streaming="aa", stats_every=4)
    g = Channel.from_case(c, check_every=5, mass_tol=0.5)
    g.step(8 + start)
    full = g.get_state()
    blk = g.get_block(3, 0, 9, 40, 16, 3)  # touches the walls and the periodic z end
    assert np.array_equal(blk, full[:, 9:12, 0:16, 3:43])
    xyz = np.array([[0, 0, 0], [63, 15, 11], [31, 7, 5], [1, 14, 0]], dtype=np.int32)
    g.set_probes(xyz)
    image = g.save()
    series = g.step_probed(3)
    u = velocity(g.populations())
    for k, (x, y, z) in enumerate(xyz):
        np.testing.assert_allclose(series[-1, k], u[:, z, y, x], rtol=1e-5, atol=1e-7)
    after = g.get_state()
    st = g.stats()
    g.load(image)  # resume from the checkpoint: the same three steps again
    g.step(3)
    assert np.array_equal(g.get_state(), after)
    st2 = g.stats()
    assert np.array_equal(st2["mean_sum"], st["mean_sum"]) and st2["n_samples"] == st["n_samples"]
    g.close()
    # a pull-scheme lattice refuses the in-place image
    p = Channel.from_case(c.with_(streaming="pull"), check_every=5, mass_tol=0.5)
    from paper_2205_02774_gb300.capi import StgError
    with pytest.raises(StgError):
        p.load(image)
    p.close()


def test_inplace_autotune_keeps_results():
    c = SMALL.with_(nx=192, ny=10, nz=24, streaming="aa", stats_every=5)
    ref, _ = _run(c, (7, 30))
    from paper_2205_02774_gb300.channel import Channel
    g = Channel.from_case(c, check_every=7, mass_tol=0.5)
    g.step(7)
    g.autotune(3)  # trial passes update the lattice in place; it is saved and put back
    st7 = g.stats()
    assert np.array_equal(g.get_state(), ref[0][0])
    g.step(30)
    st = g.stats()
    assert np.array_equal(g.get_state(), ref[1][0])
    assert np.array_equal(st["mean_sum"], ref[1][1]["mean_sum"]) and st7["step"] == 7
    g.close()


def test_inplace_batch_and_serve_members():
    from paper_2205_02774_gb300.channel import Channel
    from paper_2205_02774_gb300.serving import Batch, serve
    from workloads.serving import Job
    cs = [SMALL.with_(nx=64, ny=16, nz=12, stats_every=5, seed=3, streaming="aa"),
          SMALL.with_(nx=96, ny=12, nz=18, stats_every=10, storage="fp16sr", seed=4, streaming="aa"),
          SMALL.with_(nx=40, ny=10, nz=8, stats_every=2, seed=6)]
    refs = [_run(c, (43,))[0][0] for c in cs]
    chans = [Channel.from_case(c, check_every=7, mass_tol=0.5) for c in cs]
    chans[0].step(3)
    b = Batch()
    for ch in chans:
        b.add(ch)
    b.autotune(2)
    b.step(40)
    for ch in chans:
        b.remove(ch)
    chans[1].step(3)
    chans[2].step(3)
    for ch, (f, st) in zip(chans, refs):
        assert np.array_equal(ch.get_state(), f)
        assert np.array_equal(ch.stats()["rey_sum"], st["rey_sum"])
        ch.close()
    b.close()
    jobs = [Job(0.0, cs[0], 120), Job(0.0, cs[1], 90), Job(0.001, cs[2], 60)]
    results, rep = serve(jobs, hbm_budget_bytes=4e9, check_every=7, keep_stats=True)
    assert rep["completed"] == 3
    for jb, r in zip(jobs, results):
        (f, st), = _run(jb.case, (jb.steps,))[0]
        assert np.array_equal(r["rey_sum"], st["rey_sum"]) and r["n_samples"] == st["n_samples"]
