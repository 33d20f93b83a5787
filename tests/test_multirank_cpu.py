"""The multi-rank path on CPU (gloo, world size 2): trajectories shard across
ranks with one Philox key per rank; the bench takes the maximum of the ranks'
timed regions, and the one exchange of results (observable sums, jump
records, gradients) merges the ranks' trajectories into one ensemble."""
import os
import socket

import numpy as np
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


def _merge_rank(rank, world, port, out):
    import torch.distributed as dist

    import workloads as W
    from oracle import trajectories
    from paper_1710_03431_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inst = W.tfim_instance(2, 28, eta_g2=0.03, t_f=5.0, n_grid=31, seed=99)
        M = 6
        p, jumps, _ = trajectories.sample(inst, list(range(M)), seed=shard.rank_seed(inst.seed, rank))
        mean, se, Mt = shard.merged_observables(p.sum(axis=0), (p ** 2).sum(axis=0), M)
        from paper_1710_03431_gb300 import aqt as A
        rec = np.array([(j["traj"], j["grid"], j["half"], j["alpha"], j["src"], j["dst"], j["t"], j["omega"])
                        for j in jumps], dtype=A.JUMP_DTYPE)
        allj = shard.gather_jumps(rec, M)
        out[rank] = (p, mean, se, Mt, allj, rec)
    finally:
        dist.destroy_process_group()


def test_two_ranks_merge_observables_and_jumps(aqt_lib):
    """The merged mean and standard error equal those of one ensemble made of
    both ranks' trajectories (Eq. stderror); the gathered jump log is the
    union of the ranks' logs with rank-major trajectory indices."""
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_merge_rank, args=(2, port, out), nprocs=2, start_method="spawn")
        res = dict(out)
    p_all = np.concatenate([res[0][0], res[1][0]])
    R = len(p_all)
    mean = p_all.mean(axis=0)
    se = p_all.std(axis=0, ddof=1) / np.sqrt(R)
    for r in (0, 1):
        _, m, s, Mt, allj, _ = res[r]
        assert Mt == R
        np.testing.assert_allclose(m, mean, rtol=0, atol=1e-14)
        # the sums form (sum x^2 - R mean^2) cancels where every x is alike: an
        # absolute floor of sqrt(eps sum x^2 / (R (R - 1)))
        np.testing.assert_allclose(s, se, rtol=1e-9, atol=np.sqrt(4e-16 * R / (R - 1.0)))
    own0, own1 = res[0][5], res[1][5]
    assert len(res[0][4]) == len(own0) + len(own1) > 0
    assert np.array_equal(res[0][4], res[1][4])
    assert set(res[0][4]["traj"].tolist()) == set(own0["traj"].tolist()) | {t + 6 for t in own1["traj"].tolist()}


def _grad_rank(rank, world, port, out):
    import torch.distributed as dist

    import workloads as W
    from oracle import gradient as G
    from oracle import trajectories
    from paper_1710_03431_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inst = W.tfim_instance(2, 3, eta_g2=0.05, t_f=4.0, n_grid=6, seed=7, lamb_shift=False)
        M = 2 + rank  # uneven shards
        seed = shard.rank_seed(inst.seed, rank)
        p, jumps, _ = trajectories.sample(inst, list(range(M)), seed=seed)
        per = [G.trajectory_gradient_fd(inst, [j for j in jumps if j["traj"] == t], baseline=0.5)[0]
               for t in range(M)]
        g, Mt = shard.merge_gradient(np.mean(per, axis=0), M)
        out[rank] = (np.array(per), g, Mt)
    finally:
        dist.destroy_process_group()


def test_two_ranks_merge_gradients():
    """The merged gradient is the mean of the per-trajectory estimates of both
    ranks' trajectories (uneven shards), NaN where a parameter has none."""
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_grad_rank, args=(2, port, out), nprocs=2, start_method="spawn")
        res = dict(out)
    allper = np.concatenate([res[0][0], res[1][0]])
    ref = allper.mean(axis=0)
    for r in (0, 1):
        _, g, Mt = res[r]
        assert Mt == len(allper) == 5
        np.testing.assert_allclose(g, ref, rtol=1e-13, atol=1e-15)

