"""Multi-GPU runs are independent replicas (the path has no exchange step):
bench.py takes the slowest rank's time and counts every rank's evaluations.
Checked here with world_size 2 over the gloo backend on CPU."""
import os
import socket

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
        ms = bench.replica_max_ms(100.0 + 50.0 * rank, "cpu")
        out[rank] = (ms, bench.job_value(world, 8, 5, ms))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 150.0
        assert abs(value - world * 8 * 5 / 0.150) < 1e-9


def test_single_process_keeps_its_time():
    import bench
    assert bench.replica_max_ms(123.0, "cpu") == 123.0
    assert abs(bench.job_value(1, 8, 5, 123.0) - 8 * 5 / 0.123) < 1e-9
