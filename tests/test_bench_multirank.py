"""The multi-rank bench path (independent replicas) on CPU with two gloo ranks.

Each rank reports its own timing; the job value is every rank's work over the
slowest rank's time.  No GPU: this checks the host-side aggregation that
`bench.py --gpus N` performs under torchrun.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0, 25.0][rank]                 # rank 1 is the slow one
    out[rank] = bench.aggregate(ms, 8 * 20, dist)
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_max_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms, value = res[rank]
        assert ms == 25.0
        assert value == pytest.approx(2 * 8 * 20 / 0.025)


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate(4.0, 80) == (4.0, 80 / 0.004)
