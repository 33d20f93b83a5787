"""The trajectory average of the ground-state population at s = 1 as a
differentiable function of the annealing parameters (torch.autograd.Function).

Argument marshalling only: the forward run (with checkpoints) and the adjoint
sweep are libaqt's (aqt_grad_forward, aqt_grad_backward, aqt_grad_get; the
estimator is stated in include/aqt.h).

Parameters theta (1-D, float64), in the library's order: A(s) at the schedule
knots, B(s) at the knots, hz_i, Jzz_ij (i < j, row by row). The instance gives
everything else (knot positions, bath, grid, t_f, M, seed).
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import aqt as A


def instance_with(inst, theta: np.ndarray):
    """A copy of ``inst`` whose schedule values, fields and couplings are theta."""
    k = len(inst.sched_s)
    n = inst.n_qubits
    out = copy.deepcopy(inst)
    out.sched_A = np.array(theta[:k], dtype=np.float64)
    out.sched_B = np.array(theta[k:2 * k], dtype=np.float64)
    out.hz = np.array(theta[2 * k:2 * k + n], dtype=np.float64)
    J = np.zeros((n, n))
    J[np.triu_indices(n, k=1)] = theta[2 * k + n:]
    out.J = J
    return out


def parameters_of(inst) -> np.ndarray:
    iu = np.triu_indices(inst.n_qubits, k=1)
    return np.concatenate([np.asarray(inst.sched_A, float), np.asarray(inst.sched_B, float),
                           np.asarray(inst.hz, float), np.asarray(inst.J, float)[iu]])


class GroundPopulation(torch.autograd.Function):
    """<P_GS(s = 1)>(theta). forward: one checkpointed run of inst.M
    trajectories; backward: the adjoint sweep of that run. The derivative of a
    parameter that has none (it couples a degenerate manifold, e.g. B at s = 0)
    is NaN."""

    @staticmethod
    def forward(ctx, theta, inst, precision, seed, checkpoint_every, baseline, device):
        th = theta.detach().to("cpu", torch.float64).numpy()
        S = A.Session(instance_with(inst, th), precision=precision, seed=seed, device=device)
        S.build()
        S.grad_allocate(checkpoint_every)
        A.aqt_grad_forward(S.ctx, S.stream())
        A.aqt_sync(S.ctx)
        mean, _ = S.observables()
        ctx.session = S
        ctx.baseline = baseline
        ctx.theta_meta = (theta.dtype, theta.device)
        return torch.tensor(float(mean[-1]), dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        S = ctx.session
        try:
            A.aqt_grad_backward(S.ctx, ctx.baseline, S.stream())
            g, _ = A.aqt_grad_get(S.ctx, A.aqt_grad_n_params(S.ctx))
        finally:
            S.close()
            ctx.session = None
        dtype, dev = ctx.theta_meta
        return grad_out * torch.as_tensor(g, dtype=dtype, device=dev), None, None, None, None, None, None


def ground_population(theta, inst, precision=A.AQT_PREC_FP32, seed=None, checkpoint_every=64,
                      baseline=float("nan"), device=0):
    """<P_GS(1)> for parameters theta (see the module docstring); differentiable."""
    return GroundPopulation.apply(theta, inst, precision, seed, checkpoint_every, baseline, device)
