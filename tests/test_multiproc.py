"""The multi-process (N > 1) host logic of the benchmark on CPU with gloo, world size 2.

The data path never communicates (independent replicas); what crosses ranks is the
barrier and the max-over-ranks of the timed region, and each rank takes its own frames.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    seeds = bench.frame_seeds(rank, world, 8)
    dist.barrier()
    got = [None] * world
    dist.all_gather_object(got, seeds)
    out[rank] = (t, got)
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_disjoint_frames():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a threaded process
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, seeds = res[rank]
        assert t == 15.0
        assert set(seeds[0]).isdisjoint(seeds[1])
        assert seeds[0] == list(range(1, 9))


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
