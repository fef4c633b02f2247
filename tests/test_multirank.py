"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the job time is the
slowest rank's, and the whole-job throughput counts every rank's independent problem."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        return sck.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank          # rank 1 is slower
    t = bench.max_over_ranks(local_ms, torch.device("cpu"))
    v = bench.job_throughput(1000, 10, 2, t, world)
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        t, v = out[r]
        assert t == 150.0
        assert abs(v - 2 * 1000 * 10 * 2 / 0.150) < 1e-6


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, torch.device("cpu")) == 12.5
    assert bench.job_throughput(10, 5, 2, 1000.0, 1) == 100.0
