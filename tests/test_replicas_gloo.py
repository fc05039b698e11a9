"""The N > 1 benchmark path on CPU: two gloo ranks, independent replicas,
aggregated as (sum of units) / (max of times), with no data-path exchange."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1812_07167_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        units, ms = 1000.0 * (rank + 1), 10.0 + 5.0 * rank
        total, mx = replicas.aggregate(units, ms)
        thr = replicas.throughput(units, ms)
        out[rank] = (total, mx, thr)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:  # no fork of this multi-threaded process
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        total, mx, thr = res[rank]
        assert total == 3000.0
        assert mx == 15.0
        assert thr == pytest.approx(3000.0 / 0.015)


def test_single_process_is_identity():
    assert replicas.aggregate(5.0, 2.0) == (5.0, 2.0)
    assert replicas.throughput(5.0, 2.0) == pytest.approx(2500.0)
