"""Replica aggregation across ranks (the multi-GPU path of the benchmark),
run as two gloo ranks on CPU."""
import os
import socket

import pytest


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2108_08769_gb300.replicas import aggregate
    units, ms, rate = aggregate(100.0 * (rank + 1), 10.0 * (rank + 1))
    out[rank] = (units, ms, rate)
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_units_and_take_max_time():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, free_port(), out), nprocs=2, join=True)
    for r in range(2):
        units, ms, rate = out[r]
        assert units == 300.0 and ms == 20.0
        assert rate == pytest.approx(300.0 / 0.020)


def test_single_process_without_group():
    from paper_2108_08769_gb300.replicas import aggregate
    assert aggregate(50.0, 5.0) == (50.0, 5.0, pytest.approx(1e4))
