"""The benchmark's multi-replica aggregation on two gloo ranks (CPU): the
slowest rank's time against all ranks' cell updates."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [40.0, 55.0][rank]  # rank 1 is the slow one
    total, value = bench.aggregate(ms, 1e9, world, device="cpu")
    results[rank] = (total, value)
    dist.destroy_process_group()


def test_aggregate_takes_max_over_two_gloo_ranks():
    mgr = mp.Manager()
    results = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), results), nprocs=2, join=True)
    for rank in (0, 1):
        total, value = results[rank]
        assert total == 55.0
        assert value == pytest.approx(2 * 1e9 / 0.055 / 1e9)


def test_aggregate_single_rank():
    import bench
    total, value = bench.aggregate(20.0, 4e9, 1)
    assert total == 20.0 and value == pytest.approx(200.0)
