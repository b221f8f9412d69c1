"""The multi-rank (N > 1) path of the benchmark on CPU: two gloo ranks run
the rank aggregation that bench.py uses under torchrun (one independent
channel per GPU, no collective on the data path, max over ranks of the timed
region, sum of the cell updates)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms_local = 10.0 * (rank + 1)          # rank 1 is the slow one
        cells = 1000 * (rank + 1)             # and holds a larger channel
        out[rank] = bench.aggregate_ranks(ms_local, cells, 50, dist) + (bench.rank_seed(7, rank),)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn")
        res = dict(out)
    for r in range(ws):
        ms, value, seed = res[r]
        assert ms == pytest.approx(20.0)                       # max over ranks
        assert value == pytest.approx(3000 * 50 / 20e-3 / 1e6)  # all ranks' cell updates / max time
        assert seed == 7 + r                                    # independent channel per rank


def test_single_rank_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate_ranks(4.0, 2.0e6, 100)
    assert ms == 4.0 and value == pytest.approx(2.0e6 * 100 / 4e-3 / 1e6)


def test_launch_count_includes_statistics_reductions():
    """gpu_launches: per step the inlet kernel and the two step launches of the
    vector path, plus one statistics reduction after every sampling step
    ((t + 1) % stats_every == 0) in the timed range; the scalar path (odd nx)
    launches the inlet, interior and edge kernels and no reduction."""
    sys.path.insert(0, ROOT)
    import bench
    from workloads import case
    c = case("channel_768x128x192")
    assert c.stats_every == 10
    assert bench._launches_per_step(c) == 3
    assert bench._launches(c, 200, 4000) == 3 * 4000 + 400
    assert bench._launches(c, 5, 10) == 30 + 1            # t = 9 samples
    assert bench._launches(c.with_(stats_every=0), 5, 10) == 30
    odd = c.with_(nx=767)
    assert bench._launches(odd, 0, 20) == 3 * 20


def test_bench_variants():
    """--collision / --sponge: the paper's sponge is 0.4 delta (delta = ny / 2)
    with K = 1000 and p = 3; defaults leave the workload unchanged."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    from workloads import case
    c = case("channel_768x128x192")
    same = bench._variant(c, argparse.Namespace(collision="regularized", sponge=False))
    assert same.collision == "regularized" and same.sponge_len == 0.0
    v = bench._variant(c, argparse.Namespace(collision="bgk", sponge=True))
    assert v.collision == "bgk"
    assert abs(v.sponge_len - 0.4 * 128 / 2) < 1e-12 and v.sponge_K == 1000.0 and v.sponge_p == 3.0
    assert (v.nx, v.ny, v.nz) == (c.nx, c.ny, c.nz)
