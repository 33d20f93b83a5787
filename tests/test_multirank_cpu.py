"""The multi-rank bench path on CPU (gloo, world size 2): trajectories shard
across ranks with one Philox key per rank and no data-path collective; the
only exchange is the maximum of the ranks' timed regions."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench
from oracle import philox


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = (bench.max_over_ranks(1.5 + rank), bench.rank_seed(1710_03432, rank))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_distinct_streams():
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    s0, s1 = res[0][1], res[1][1]
    assert s0 != s1
    # independent streams: the first thresholds of the same trajectory index differ
    assert philox.first_threshold(s0, 0) != philox.first_threshold(s1, 0)
