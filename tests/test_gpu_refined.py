"""The refined channel (h = 128, 1536 x 256 x 384, 151M cells) in FP32 and in
shifted-FP16 storage: one step from the GPU's own state checked cell by cell
against the oracle on a 64^3 sub-block (the oracle reads the sub-block and a
one-cell halo), and the FP16 run's mean and Reynolds-stress sums against the
FP32 run's after 200 steps (within 1 %, normwise)."""
import numpy as np
import pytest

from workloads import case

from gpu_helpers import require_cuda, normwise, fp16_half_ulp, W19

pytestmark = pytest.mark.gpu

REFINED = case("channel_1536x256x384")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
def test_refined_subblock_one_step(storage):
    import oracle as O
    from paper_2205_02774_gb300.channel import Channel
    c = REFINED.with_(storage=storage)
    g = Channel.from_case(c, check_every=10, mass_tol=0.1)
    g.step(3)
    x0, y0, z0, n = 700, 96, 150, 64
    pre = g.get_block(x0 - 1, y0 - 1, z0 - 1, n + 2, n + 2, n + 2)
    g.step(1)
    post = g.get_block(x0, y0, z0, n, n, n)
    st = g.stats()
    g.close()
    assert st["rc"] == 0, st["error"]
    # the block with its halo as a lattice of its own: interior cells only read inside it
    dom = O.make_domain(n + 2, n + 2, n + 2, c.tau0, c.c_smag, c.force, "periodic", "periodic", c.collision)
    if storage == "fp32":
        got = post.astype(np.float64) + W19.reshape(19, 1, 1, 1)
    else:
        got = post.view(np.float16).astype(np.float64) + W19.reshape(19, 1, 1, 1)
    worst = 0.0
    for z in range(n):
        for y in range(n):
            for x in range(n):
                ref = O.cell_update(dom, pre, x + 1, y + 1, z + 1, shifted=True)
                v = got[:, z, y, x]
                if storage == "fp32":
                    worst = max(worst, float(np.max(np.abs(v - ref) / np.abs(ref))))
                else:
                    bound = fp16_half_ulp(ref - W19) + 2e-6 * np.abs(ref)
                    worst = max(worst, float(np.max(np.abs(v - ref) - bound)))
    if storage == "fp32":
        assert worst < 1e-5
    else:
        assert worst <= 0


def test_refined_fp16_profiles_vs_fp32():
    from paper_2205_02774_gb300.channel import Channel
    out = {}
    for storage in ("fp32", "fp16s"):
        g = Channel.from_case(REFINED.with_(storage=storage), check_every=50, mass_tol=0.1)
        g.step(200)
        st = g.stats()
        g.close()
        assert st["rc"] == 0, st["error"]
        assert st["n_samples"] == 20
        out[storage] = st
    assert normwise(out["fp16s"]["mean_sum"], out["fp32"]["mean_sum"]) < 1e-2
    assert normwise(out["fp16s"]["rey_sum"], out["fp32"]["rey_sum"]) < 1e-2
