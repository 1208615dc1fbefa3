"""Host logic of bench.py's multi-replica path on CPU: two gloo ranks, the
slowest rank's time is the job's time and the rate counts every replica's
work."""
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
    ms = [120.0, 250.0][rank]
    slowest = bench.max_over_ranks(ms)
    out[rank] = (slowest, bench.job_throughput(1000.0, world, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 250.0
    assert out[0][1] == pytest.approx(2 * 1000.0 / 0.25)


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(10.0, 1, 1000.0) == 10.0
