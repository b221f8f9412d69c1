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
