"""Sponge zone of eq. (sponge_visco) on the GPU against the oracle.

The zone scales the relaxation of the last sponge_len columns before the
outlet; the tests cover the vector kernels (even nx, every tile; the outlet
node, rebuilt in the vector kernel, lies inside the zone), the scalar kernels
(odd nx) and a periodic-x lattice with the zone over part of x.
"""
import numpy as np
import pytest

from workloads import case, perturbed_equilibrium_field

from gpu_helpers import require_cuda, pair, max_rel, normwise, velocity

pytestmark = pytest.mark.gpu

SMALL = case("channel_64x32x32")
PAPER_SPONGE = dict(sponge_K=1000.0, sponge_p=3.0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


@pytest.mark.parametrize("dims,kw", [
    ((64, 10, 9), dict(sponge_len=12.8)),
    ((37, 10, 9), dict(sponge_len=9.0)),                                    # odd nx: scalar kernels
    ((200, 6, 5), dict(sponge_len=40.0, collision="bgk")),
    ((64, 8, 6), dict(sponge_len=20.0, bc_x="periodic", collision="bgk")),  # zone inside a periodic x
    ((130, 9, 11), dict(sponge_len=25.0, storage="fp16s")),
])
def test_sponge_single_step(dims, kw):
    nx, ny, nz = dims
    c = SMALL.with_(nx=nx, ny=ny, nz=nz, stats_every=0, **PAPER_SPONGE, **kw)
    gpu, orc = pair(c)
    st = gpu.encode(perturbed_equilibrium_field(nx, ny, nz, seed=nx + 2 * ny))
    gpu.set_state(st, 0)
    orc.set_pops(gpu.decode(st))
    gpu.step(1)
    orc.step(1)
    if c.storage == "fp32":
        assert max_rel(gpu.populations(), orc.pops()) < 1e-5
    else:
        from gpu_helpers import fp16_half_ulp, W19
        fo = orc.pops()
        bound = fp16_half_ulp(fo - W19.reshape(19, 1, 1, 1)) + 2e-6 * np.abs(fo)
        assert (np.abs(gpu.populations() - fo) - bound).max() <= 0


def test_sponge_channel_200_steps():
    c = SMALL.with_(sponge_len=12.8, **PAPER_SPONGE)
    gpu, orc = pair(c, check_every=20, mass_tol=0.1)
    gpu.step(c.steps)
    orc.step(c.steps)
    fg, fo = gpu.populations(), orc.pops()
    assert normwise(velocity(fg), velocity(fo)) < 1e-4
    st = gpu.stats()
    assert st["rc"] == 0, st["error"]
    m, r, n = orc.stats()
    assert st["n_samples"] == n
    assert normwise(st["mean_sum"], m) < 1e-4
    assert normwise(st["rey_sum"], r) < 1e-4


def test_sponge_tiles_bit_identical():
    from paper_2205_02774_gb300.channel import Channel
    c = SMALL.with_(nx=200, ny=10, nz=21, stats_every=3, sponge_len=30.0, **PAPER_SPONGE)
    ref = None
    for tile in [(1, 8, 24), (0, 4, 4), (1, 12, 0)]:
        g = Channel.from_case(c, check_every=5, mass_tol=0.5)
        g.set_tile(*tile)
        g.step(12)
        f, st = g.get_state(), g.stats()
        g.close()
        if ref is None:
            ref = (f, st)
        assert np.array_equal(f, ref[0]) and np.array_equal(st["rey_sum"], ref[1]["rey_sum"])


def test_sponge_rejected_with_force():
    from paper_2205_02774_gb300.capi import StgError
    from paper_2205_02774_gb300.channel import Channel
    with pytest.raises(StgError):
        Channel.from_case(SMALL.with_(bc_x="periodic", force=(1e-6, 0.0, 0.0), sponge_len=8.0))


def test_probes_match_state_and_oracle():
    """Velocity probes (step_probed) against the velocity of the stored state
    read back after the same steps, and against the oracle's run."""
    from gpu_helpers import velocity
    c = SMALL.with_(stats_every=0, sponge_len=12.8, **PAPER_SPONGE)
    gpu, orc = pair(c)
    xyz = np.array([[0, 3, 1], [5, 16, 7], [32, 0, 31], [63, 31, 0], [60, 10, 12]])
    gpu.set_probes(xyz)
    u = gpu.step_probed(5)
    assert u.shape == (5, len(xyz), 3)
    f = gpu.populations()
    ug = velocity(f)
    for k, (x, y, z) in enumerate(xyz):
        np.testing.assert_allclose(u[-1, k], ug[:, z, y, x], rtol=0, atol=1e-6)
    orc.step(5)
    uo = velocity(orc.pops())
    ref = np.array([uo[:, z, y, x] for x, y, z in xyz])
    assert np.abs(u[-1] - ref).max() <= 1e-5 * np.abs(uo).max()
    gpu.step(3)  # plain steps still work after probing
    assert gpu.stats()["rc"] == 0
