"""Failure detection and checkpoint/resume (GPU, through the C ABI).

Failures are made on the host: a NaN written by a host copy into a tiny
lattice, or a mass tolerance that a legitimate inlet/outlet run exceeds; no
GPU fault, trap or hang is involved.  The device side only computes the FP64
mass; the host reads it and reports STG_ERR_UNSTABLE."""
import numpy as np
import pytest

from workloads import case, perturbed_equilibrium_field

from gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu

SMALL = case("channel_64x32x32")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


def _poisoned(ch, seed=1):
    st = ch.encode(perturbed_equilibrium_field(ch.nx, ch.ny, ch.nz, seed=seed))
    bad = st.copy()
    if bad.dtype == np.float32:
        bad[3, 1, 2, 3] = np.nan
    else:
        bad[3, 1, 2, 3] = np.uint16(0x7E00)  # binary16 NaN
    return st, bad


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
def test_nan_is_reported_and_sticky(storage):
    from paper_2205_02774_gb300.capi import StgError, STG_ERR_UNSTABLE
    from paper_2205_02774_gb300.channel import Channel
    c = SMALL.with_(nx=16, ny=6, nz=5, storage=storage, stats_every=0)
    ch = Channel.from_case(c, check_every=5, mass_tol=0.5)
    good, bad = _poisoned(ch)
    ch.set_state(bad, 0)
    ch.step(10)
    st = ch.stats()
    assert st["rc"] == STG_ERR_UNSTABLE
    with pytest.raises(StgError) as e:
        ch.step(1)
    assert e.value.code == STG_ERR_UNSTABLE
    ch.set_state(good, 0)  # a clean state clears the error
    ch.step(10)
    assert ch.stats()["rc"] == 0
    ch.close()


def test_mass_drift_beyond_tolerance():
    from paper_2205_02774_gb300.capi import STG_ERR_UNSTABLE
    from paper_2205_02774_gb300.channel import Channel
    # an inlet/outlet channel exchanges mass through its open ends: far above 1e-12
    ch = Channel.from_case(SMALL.with_(stats_every=0), check_every=10, mass_tol=1e-12)
    ch.step(40)
    st = ch.stats()
    assert st["rc"] == STG_ERR_UNSTABLE
    assert "drift" in st["error"]
    ch.close()
    ok = Channel.from_case(SMALL.with_(stats_every=0), check_every=10, mass_tol=0.5)
    ok.step(40)
    assert ok.stats()["rc"] == 0
    ok.close()


def test_batch_reports_the_failed_member_and_continues():
    from paper_2205_02774_gb300.capi import StgError, STG_ERR_UNSTABLE
    from paper_2205_02774_gb300.channel import Channel
    from paper_2205_02774_gb300.serving import Batch
    c = SMALL.with_(nx=16, ny=6, nz=5, stats_every=0)
    a = Channel.from_case(c, check_every=4, mass_tol=0.5)
    b = Channel.from_case(c.with_(seed=3), check_every=4, mass_tol=0.5)
    _, bad = _poisoned(b)
    b.set_state(bad, 0)
    bt = Batch()
    bt.add(a)
    bt.add(b)
    bt.step(20)
    bt.sync()
    with pytest.raises(StgError) as e:
        bt.step(20)
    assert e.value.code == STG_ERR_UNSTABLE and "member 1" in str(e.value)
    bt.remove(b)
    bt.step(20)  # the healthy member carries on
    bt.sync()
    assert a.stats()["rc"] == 0 and a.stats()["step"] == 40
    bt.close()
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
def test_checkpoint_resume_bit_identical(storage):
    from paper_2205_02774_gb300.capi import StgError
    from paper_2205_02774_gb300.channel import Channel
    c = SMALL.with_(storage=storage, stats_every=5)
    a = Channel.from_case(c, check_every=7, mass_tol=0.5)
    a.step(33)
    image = a.save()
    a.step(27)
    ref_f, ref_s = a.get_state(), a.stats()
    b = Channel.from_case(c, check_every=7, mass_tol=0.5)
    b.step(4)  # some other state, overwritten by the load
    b.load(image)
    b.step(27)
    f, s = b.get_state(), b.stats()
    assert np.array_equal(f, ref_f)
    assert np.array_equal(b.inlet(), a.inlet())
    assert np.array_equal(s["mean_sum"], ref_s["mean_sum"]) and np.array_equal(s["rey_sum"], ref_s["rey_sum"])
    assert s["n_samples"] == ref_s["n_samples"] and s["step"] == ref_s["step"] == 60
    other = Channel.from_case(c.with_(nx=32), check_every=7, mass_tol=0.5)
    with pytest.raises(StgError):
        other.load(image)
    for ch in (a, b, other):
        ch.close()
