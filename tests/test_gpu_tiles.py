"""Launch tiles and the autotuner (GPU, through the C ABI).

The tile of the plain step launches (warp layout and z chunk per block) only
changes how the lattice is cut into thread blocks; every tile must give
bit-identical populations and statistics, the tiled path must match the
oracle like the default one, and autotuning must leave the run's results
unchanged."""
import numpy as np
import pytest

from workloads import case, perturbed_equilibrium_field

from gpu_helpers import require_cuda, pair, max_rel

pytestmark = pytest.mark.gpu

SMALL = case("channel_64x32x32")
TILES = [(1, 8, 24), (0, 0, 0), (0, 4, 4), (1, 4, 0), (1, 12, 5), (0, 16, 8), (1, 6, 24)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def _run(c, tile, steps, **kw):
    from paper_2205_02774_gb300.channel import Channel
    g = Channel.from_case(c, **kw)
    if tile is not None:
        g.set_tile(*tile)
        assert g.tile() == tuple(tile)
    g.step(steps)
    st = g.stats()
    f = g.get_state()
    g.close()
    assert st["rc"] == 0, st["error"]
    return f, st


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
@pytest.mark.parametrize("variant", ["channel", "periodic_bgk_force"])
def test_tiles_bit_identical(storage, variant):
    # nz = 37: ragged z chunks for every chunk length; nx = 200: a partial
    # 256-cell layout-1 block; stats every 3 steps mixes sampling and plain steps
    c = SMALL.with_(storage=storage, nx=200, ny=10, nz=37, stats_every=3)
    if variant == "periodic_bgk_force":
        c = c.with_(bc_x="periodic", collision="bgk", force=(2e-6, 0.0, 1e-6))
    ref = None
    for tile in TILES:
        f, st = _run(c, tile, 25, check_every=7, mass_tol=0.5)
        if ref is None:
            ref = (f, st)
            continue
        assert np.array_equal(f, ref[0]), tile
        assert np.array_equal(st["mean_sum"], ref[1]["mean_sum"]), tile
        assert np.array_equal(st["rey_sum"], ref[1]["rey_sum"]), tile
        assert abs(st["mass"] - ref[1]["mass"]) <= 1e-12 * abs(ref[1]["mass"]), tile


@pytest.mark.parametrize("tile", [(0, 4, 4), (1, 4, 0), (1, 12, 5)])
def test_tile_single_step_vs_oracle(tile):
    c = SMALL.with_(stats_every=0, nx=130, ny=9, nz=11)
    gpu, orc = pair(c)
    gpu.set_tile(*tile)
    st = gpu.encode(perturbed_equilibrium_field(c.nx, c.ny, c.nz, seed=11))
    gpu.set_state(st, 0)
    orc.set_pops(gpu.decode(st))
    gpu.step(1)
    orc.step(1)
    assert max_rel(gpu.populations(), orc.pops()) < 1e-5


def test_set_tile_rejects_bad_tiles():
    from paper_2205_02774_gb300.capi import StgError
    from paper_2205_02774_gb300.channel import Channel
    g = Channel.from_case(SMALL.with_(nx=64, ny=8, nz=8))
    for bad in [(2, 8, 24), (1, 2, 24), (1, 8, 3), (-1, 0, 0)]:
        with pytest.raises(StgError):
            g.set_tile(*bad)
        assert g.tile() == (1, 8, 24)
    g.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
def test_autotune_leaves_results_unchanged(storage):
    from paper_2205_02774_gb300.channel import Channel
    c = SMALL.with_(storage=storage, nx=128, ny=12, nz=20, stats_every=5)
    a = Channel.from_case(c, check_every=4, mass_tol=0.5)
    b = Channel.from_case(c, check_every=4, mass_tol=0.5)
    a.step(9)
    b.step(9)  # the next step (t = 9) is a sampling and a check step
    chosen = b.autotune(3)
    assert b.tile() == chosen
    assert chosen[0] in (0, 1)
    a.step(13)
    b.step(13)
    sa, sb = a.stats(), b.stats()
    assert sa["rc"] == 0 and sb["rc"] == 0
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(sa["mean_sum"], sb["mean_sum"])
    assert np.array_equal(sa["rey_sum"], sb["rey_sum"])
    assert sa["n_samples"] == sb["n_samples"]
    a.close()
    b.close()
