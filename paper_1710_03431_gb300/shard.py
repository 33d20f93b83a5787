"""Trajectories sharded over several GPUs (one process and one context per
GPU): the one exchange step of the path.

Trajectories are independent (Sec. VI.C), so each rank runs its own M_r
trajectories with its own Philox key (seed + rank) and no data crosses ranks
during a run. Afterwards the per-grid FP64 sums (sum x, sum x^2) add across
ranks (one all-reduce of 2 n_grid + 1 doubles) and the library turns the
merged sums into the mean and standard error (aqt_observables_from_sums,
Eq. stderror); jump records are gathered with the trajectory index made
global (rank r's trajectory t is r * M_r + t when every rank runs M_r).
torch.distributed is the transport (NCCL on GPUs, gloo on CPU); nothing here
does the method's arithmetic.
"""
from __future__ import annotations

import numpy as np

from . import aqt as A


def rank_seed(base: int, rank: int) -> int:
    """Philox key of a rank's trajectories: seed + rank."""
    return base + rank


def merge_sums(sum_x, sum_x2, M_local: int, group=None, device=None):
    """All-reduce (sum) of the ranks' observable sums and trajectory counts.
    Returns (sum_x, sum_x2, M_total) as numpy FP64 arrays and an int."""
    import torch
    import torch.distributed as dist
    K = len(sum_x)
    buf = torch.empty(2 * K + 1, dtype=torch.float64, device=device)
    buf[:K] = torch.as_tensor(np.asarray(sum_x, dtype=np.float64))
    buf[K:2 * K] = torch.as_tensor(np.asarray(sum_x2, dtype=np.float64))
    buf[2 * K] = float(M_local)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    out = buf.cpu().numpy()
    return out[:K].copy(), out[K:2 * K].copy(), int(round(out[2 * K]))


def merged_observables(sum_x, sum_x2, M_local: int, group=None, device=None):
    """Mean and standard error over the trajectories of every rank."""
    s1, s2, M = merge_sums(sum_x, sum_x2, M_local, group, device)
    mean, se = A.aqt_observables_from_sums(M, s1, s2)
    return mean, se, M


def gather_jumps(jumps: np.ndarray, M_local: int, group=None):
    """Every rank's jump records (aqt_get_jumps arrays) on every rank, with
    trajectory indices made global (rank-major), sorted by (traj, t)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = jumps.copy()
    mine["traj"] += rank * M_local
    parts = [None] * world
    dist.all_gather_object(parts, mine, group=group)
    allj = np.concatenate(parts) if parts else mine
    order = np.lexsort((allj["t"], allj["traj"]))
    return allj[order]


def merge_gradient(grad, M_local: int, group=None, device=None):
    """The gradient of the merged ensemble from the ranks' gradients (each the
    mean over its own M_r trajectories, aqt_grad_get): one all-reduce (sum) of
    M_r grad_r and M_r; the merged value is their ratio. A parameter without a
    derivative (NaN) stays NaN. Returns (grad, M_total)."""
    import torch
    import torch.distributed as dist
    g = np.asarray(grad, dtype=np.float64)
    buf = torch.empty(len(g) + 1, dtype=torch.float64, device=device)
    buf[:len(g)] = torch.as_tensor(g * float(M_local))
    buf[len(g)] = float(M_local)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    out = buf.cpu().numpy()
    M = out[len(g)]
    return out[:len(g)] / M, int(round(M))

