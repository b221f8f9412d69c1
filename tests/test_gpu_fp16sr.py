"""Shifted binary16 storage written by stochastic rounding (STG_FP16_SHIFTED_SR).

A stored population is one of the two binary16 neighbours of the FP32
result, the upper one with probability equal to the result's distance from
the lower one in units of their spacing, so it is within one spacing of the
oracle and unbiased.  Round to nearest drops every update smaller than half
a spacing: in a slowly driven flow it stagnates, stochastic rounding keeps
the update on average.  The random bits are a fixed function of cell, step
and population, so runs are reproducible."""
import numpy as np
import pytest

from workloads import case, perturbed_equilibrium_field

from gpu_helpers import require_cuda, pair, velocity, fp16_bits, fp16_decode, W19

pytestmark = pytest.mark.gpu

SMALL = case("channel_64x32x32")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def _spacing(vals):
    return np.spacing(np.abs(vals).astype(np.float16)).astype(np.float64)


@pytest.mark.parametrize("dims,kw", [((64, 32, 32), dict()), ((101, 5, 7), dict()),
                                     ((130, 6, 5), dict(bc_x="periodic", force=(2e-5, 0.0, 1e-5))),
                                     ((66, 10, 7), dict(streaming="aa")), ((66, 10, 7), dict()),
                                     ((136, 6, 5), dict(bc_x="periodic")), ((136, 6, 5), dict(bc_x="periodic", streaming="aa"))])
def test_fp16sr_single_step_within_one_spacing(dims, kw):
    nx, ny, nz = dims
    c = SMALL.with_(nx=nx, ny=ny, nz=nz, stats_every=0, storage="fp16sr", **kw)
    gpu, orc = pair(c, **({"streaming": kw["streaming"]} if "streaming" in kw else {}))
    bits = fp16_bits(perturbed_equilibrium_field(nx, ny, nz, seed=8))
    gpu.set_state(bits, 0)
    orc.set_pops(fp16_decode(bits))
    gpu.step(1)
    orc.step(1)
    fo = orc.pops()
    W = W19.reshape(19, 1, 1, 1)
    err = fp16_decode(gpu.get_state()) - fo
    assert (np.abs(err) - (_spacing(fo - W) + 2e-6 * np.abs(fo))).max() <= 0
    # unbiased: the mean error in units of the spacing vanishes (RN's would too,
    # but SR's errors spread over the whole spacing, not half of it)
    z = err / _spacing(fo - W)
    assert abs(z.mean()) < 5 * z.std() / np.sqrt(z.size)
    assert np.abs(z).max() > 0.6


def test_fp16sr_keeps_small_updates():
    """Force-driven periodic box at rest: each step adds F to the momentum of
    every cell (Guo forcing), an update far below half a binary16 spacing of
    the populations it changes.  After n steps the mean velocity is (n - 1/2) F
    in FP32 storage; round to nearest keeps it at zero, stochastic rounding
    reaches (n - 1/2) F on average."""
    from paper_2205_02774_gb300.channel import Channel
    F, n = 2e-8, 400
    res = {}
    for storage in ("fp32", "fp16s", "fp16sr"):
        g = Channel(32, 32, 32, tau0=0.8, c_smag=0.0, force=(F, 0.0, 0.0), bc_x="periodic", bc_y="periodic",
                    storage=storage)
        g.step(n)
        res[storage] = velocity(g.populations(), (F, 0.0, 0.0))[0].mean()
        g.close()
    exact = (n - 0.5) * F
    assert res["fp32"] == pytest.approx(exact, rel=1e-4)
    assert abs(res["fp16s"]) < 0.05 * exact            # stagnation
    assert res["fp16sr"] == pytest.approx(exact, rel=0.05)


def test_fp16sr_reproducible_and_tile_independent():
    from paper_2205_02774_gb300.channel import Channel
    c = SMALL.with_(nx=256, ny=12, nz=20, storage="fp16sr", stats_every=5)
    out = []
    for tile in ((1, 8, 24), (0, 16, 4), (1, 4, 24)):
        g = Channel.from_case(c, check_every=7, mass_tol=0.5)
        g.set_tile(*tile)
        g.step(23)
        out.append((g.get_state(), g.stats()["rey_sum"]))
        g.close()
    for f, r in out[1:]:
        assert np.array_equal(f, out[0][0]) and np.array_equal(r, out[0][1])
