"""The allocation-free mass entry point against the existing one.

stg_lattice_mass_noalloc serves callers that cannot allocate device memory;
it runs the mass reduction with its scratch in a static device array.  Its
result must equal the mass that stg_lbm_stats reports for the same state, on
two calls in a row (the second call reuses the scratch the first one left).
This file is collected last so that a failure here does not hide the others.
"""
import pytest

from workloads import case

from gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
def test_noalloc_mass_matches_stats(storage):
    torch = require_cuda()
    from paper_2205_02774_gb300 import capi
    from paper_2205_02774_gb300.channel import Channel
    c = case("channel_64x32x32").with_(storage=storage, stats_every=0)
    ch = Channel.from_case(c)
    code = capi.STG_FP32 if storage == "fp32" else capi.STG_FP16_SHIFTED
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for steps in (5, 3):
        ch.step(steps)
        ref = ch.stats()
        assert ref["rc"] == 0, ref["error"]
        pops, _ = ch.device_state()
        for _ in range(2):
            out.fill_(-1.0)
            rc = capi.stg_lattice_mass_noalloc(pops, code, c.nx, c.ny, c.nz, out.data_ptr(), ch.stream.cuda_stream)
            assert rc == capi.STG_OK, capi.stg_lbm_last_error()
            ch.stream.synchronize()
            assert abs(out.item() - ref["mass"]) <= 1e-12 * abs(ref["mass"])
    ch.close()


def test_noalloc_mass_rejects_bad_sizes():
    torch = require_cuda()
    from paper_2205_02774_gb300 import capi
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    src = torch.zeros(19 * 8, dtype=torch.float32, device="cuda")
    rc = capi.stg_lattice_mass_noalloc(src.data_ptr(), capi.STG_FP32, 2048, 2048, 1024, out.data_ptr(), 0)
    assert rc == capi.STG_ERR_INVALID
    assert "2^31-1" in capi.stg_lbm_last_error()
    rc = capi.stg_lattice_mass_noalloc(src.data_ptr(), 7, 2, 2, 2, out.data_ptr(), 0)
    assert rc == capi.STG_ERR_INVALID
