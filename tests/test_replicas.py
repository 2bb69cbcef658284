"""Multi-process replica timing of bench.py on CPU (gloo, world size 2).

bench.py runs one independent replica per GPU; the job is timed by its
slowest replica and its throughput is the sum over replicas.  The collective
and the arithmetic are checked here with two CPU ranks over gloo.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r took 100 + 50 r ms for its 3 solves of 12 x 12 systems
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, world, torch.device("cpu"))
        out[rank] = (ms, bench.replica_value(world, 12, 12, 3, ms / 1e3))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_timed_by_slowest_rank():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 150.0                       # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 12 * 12 * 3 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(42.5, 1, torch.device("cpu")) == 42.5
    assert bench.replica_value(1, 12, 12, 5, 2.0) == pytest.approx(360.0)
