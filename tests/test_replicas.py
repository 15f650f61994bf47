"""Replica aggregation of bench.py across ranks (gloo, world size 2, CPU).

The solve does not shard inside one GPU's problem, so N > 1 runs N
independent replicas; the bench reports the slowest rank's time and the
whole job's time per solve.  This runs that arithmetic through a real
two-process gloo group."""
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
        local_ms = [120.0, 150.0][rank]          # the ranks' own timed regions
        tmax = bench.max_over_ranks(local_ms, world, dist, "cpu")
        out[rank] = (tmax, bench.job_ms_per_solve(tmax, 10, world))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        tmax, per_solve = out[r]
        assert tmax == 150.0                        # every rank sees the slowest time
        assert per_solve == pytest.approx(150.0 / (10 * 2))   # 20 solves in 150 ms


def test_single_rank_is_its_own_time():
    assert bench.max_over_ranks(7.5, 1, None, "cpu") == 7.5
    assert bench.job_ms_per_solve(100.0, 20, 1) == 5.0


def test_roofline_traffic_comes_from_committed_profiles():
    # the bench's `roofline.traffic` of each form's dominant kernel class is
    # read from a committed ncu summary measured at the headline size
    for form, name in bench.SMOOTH_PROFILE.items():
        assert name.endswith("512x128x400.md"), name
        t = bench.traffic_from_profile(name)
        assert t is not None and 1e8 < t < 1e9, (form, name, t)
    assert bench.traffic_from_profile("no_such_profile.md") is None
