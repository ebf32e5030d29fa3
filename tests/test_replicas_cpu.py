"""Replica timing over ranks (the multi-GPU launch of the benchmark runs
independent replicas: no collective on the data path, one max-reduction of
the step times).  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: step time 1 + r, host time 3 - r
        t_step, t_host = bench.reduce_replicas([1.0 + rank, 3.0 - rank], dist)
        out[rank] = (t_step, t_host, world / t_step)
    finally:
        dist.destroy_process_group()


def test_reduce_replicas_single_process():
    assert bench.reduce_replicas([0.5, 0.25]) == [0.5, 0.25]


@pytest.mark.timeout(120)
def test_reduce_replicas_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        t_step, t_host, value = out[r]
        assert t_step == 2.0 and t_host == 3.0      # max over the two ranks
        assert value == pytest.approx(1.0)          # 2 replicas / 2 s
