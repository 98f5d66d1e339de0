"""The multi-GPU mode is replicas only (one independent copy of the workload
per rank, no data-path collective): bench.py takes the slowest rank's time and
reports the whole job's rate.  This checks that host logic with two gloo ranks
on the CPU (127.0.0.1 rendezvous)."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    m = bench.max_over_ranks(torch, dist, ms, "cpu")
    rate = bench.replica_rate(1000, 10, m, world)
    out[rank] = (m, rate)
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_the_work():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    m, rate = res[0]
    assert m == 20.0
    assert rate == pytest.approx(4.0 * 1000 * 10 * world / 20e-3, rel=1e-15)
