"""Multi-rank host logic of bench.py on CPU: two gloo ranks (replicas of the pass, one per GPU
in a real run) agree on the slowest rank's time and on the whole-job throughput."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [12.5, 20.0][rank]
    ms = bench.slowest_rank_ms(ms_local, torch.device("cpu"))
    out[rank] = (ms, bench.job_throughput(1000.0, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time_and_job_throughput():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 20.0
    assert value == pytest.approx(2 * 1000.0 / 0.020)


def test_single_process_passthrough():
    import bench
    assert bench.slowest_rank_ms(7.0, torch.device("cpu")) == 7.0
    assert bench.job_throughput(10.0, 1, 5.0) == pytest.approx(2000.0)
