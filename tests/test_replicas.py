"""The multi-GPU form is replicas only: N independent systems, no collective
on the data path.  Its host logic is the whole-job reduction of bench.py
(units summed over the ranks, time of the slowest rank), checked here on two
gloo ranks on the CPU."""

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
    import bench
    # rank r: 1.5 + r seconds for 10 (r + 1) units
    t, u = bench.whole_job(1.5 + rank, 10 * (rank + 1), world, "cpu")
    out[rank] = (t, u)
    dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # every rank sees the slowest rank's time and the sum of the units
    assert res[0] == res[1] == (2.5, 30.0)


def test_whole_job_single_rank_is_the_rank_itself():
    import bench
    assert bench.whole_job(3.0, 7, 1, "cpu") == (3.0, 7.0)
