"""Parameter derivatives of the trajectory average (FP64, by finite differences).

Test infrastructure only (see the package docstring).

The paper has no derivatives; these functions state what a gradient of its
method is, so that an adjoint computation can be checked against them.

Parameters theta of an instance, in this order:
    A(s) at the schedule knots, B(s) at the schedule knots (Sec. V, Eq. H_S,
    piecewise linear between knots), hz_i (i = 0..n-1), J_ij (i < j, row by row).

Observable: the ground-manifold population of H_S(1), <P_GS(1)>.

1. ``ame_gradient_fd``: central differences of the split-exact density-matrix
   AME (``ame.run``) in each parameter. The derivative of the trajectory
   average is the derivative of this density matrix (App. B.2: the trajectories
   average to it exactly on the same split).

2. ``trajectory_gradient_fd``: the per-trajectory estimate whose average is that
   derivative. A trajectory's record (jump times and channels) has probability
   density |psi~_T|^2, the squared norm of the unnormalised state built from
   the record (the no-jump propagators between jumps and each channel's jump
   operator A_i at its time, Sec. IV, Eq. jump, App. B.1 Eq. Pi(t): the
   waiting-time density times Pi_i is |A_i psi~(t)|^2). Hence
       <P_GS> = integral over records of <psi~_T|P|psi~_T>,
   and with the record held fixed,
       d<P_GS>/dtheta = E[ d<psi~_T|P - b|psi~_T>/dtheta / |psi~_T|^2 ]
                      = E[ dp/dtheta + (p - b) d log|psi~_T|^2 / dtheta ],
   p = <psi_T|P|psi_T> of the normalised final state; b is any constant (it
   multiplies the score d log|psi~_T|^2, whose mean is zero). The first term is
   the pathwise derivative between and through the jumps at fixed jump times;
   the second is the score of the record: of the waiting-time densities and of
   the channel probabilities. This function replays a record at theta +- delta
   (same times, same channels: qubit alpha, source and target manifolds) in
   the computational basis with scipy matrix exponentials and differences
   p and log|psi~_T|^2.
"""
from __future__ import annotations

import copy

import numpy as np
from scipy import linalg

from . import ame, model


def n_params(inst) -> int:
    n = inst.n_qubits
    return 2 * len(inst.sched_s) + n + n * (n - 1) // 2


def param_vector(inst) -> np.ndarray:
    iu = np.triu_indices(inst.n_qubits, k=1)
    return np.concatenate([np.asarray(inst.sched_A, float), np.asarray(inst.sched_B, float),
                           np.asarray(inst.hz, float), np.asarray(inst.J, float)[iu]])


def with_params(inst, theta) -> object:
    """A copy of ``inst`` with the parameters theta."""
    theta = np.asarray(theta, float)
    k = len(inst.sched_s)
    n = inst.n_qubits
    out = copy.deepcopy(inst)
    out.sched_A = theta[:k].copy()
    out.sched_B = theta[k:2 * k].copy()
    out.hz = theta[2 * k:2 * k + n].copy()
    J = np.zeros((n, n))
    J[np.triu_indices(n, k=1)] = theta[2 * k + n:]
    out.J = J
    return out


def _bumped(inst, i: int, h: float):
    th = param_vector(inst)
    th[i] += h
    return with_params(inst, th)


def ame_gradient_fd(inst, delta: float = 1e-4, which=None) -> np.ndarray:
    """Central differences (step delta) of the split-exact AME's final
    ground-manifold population in the parameters ``which`` (default all)."""
    which = range(n_params(inst)) if which is None else which
    out = np.full(n_params(inst), np.nan)
    for i in which:
        hi = ame.run(_bumped(inst, i, delta))["p_gs"][-1]
        lo = ame.run(_bumped(inst, i, -delta))["p_gs"][-1]
        out[i] = (hi - lo) / (2.0 * delta)
    return out


def replay(inst, jumps):
    """Rebuild one trajectory from its record (jump dicts of ``trajectories.sample``
    for that trajectory) on the instance's frames: the no-jump propagator
    exp(-i H_eff t) of each frozen piece between the recorded times, and at each
    record the operator of its channel (qubit alpha, the Bohr class of the pair
    (target manifold, source manifold)) applied unnormalised.

    Returns (p, log_norm2): the final ground-manifold population of the
    normalised state and log |psi~_T|^2 of the unnormalised one."""
    s_grid, dt = model.grid(inst)
    tau = 0.5 * dt
    by_piece = {}
    for j in sorted(jumps, key=lambda r: r["t"]):
        by_piece.setdefault((j["grid"], j["half"]), []).append(j)
    psi = None
    logn = 0.0
    prev = None

    def piece(fr, g, half, t0, psi, logn):
        V = fr.eig.V
        Heff = V @ fr.K @ V.T
        elapsed = 0.0
        for j in by_piece.get((g, half), []):
            t = j["t"] - t0
            psi = linalg.expm(-1j * Heff * (t - elapsed)) @ psi
            elapsed = t
            a = int(j["dst"])
            b = int(j["src"])
            cls = fr.class_of_pair[a, b]
            A = np.where(fr.class_of_pair == cls, fr.R[int(j["alpha"])], 0.0)
            psi = V @ (A @ (V.T @ psi))
            nrm = np.linalg.norm(psi)
            logn += 2.0 * np.log(nrm)
            psi = psi / nrm
        psi = linalg.expm(-1j * Heff * (tau - elapsed)) @ psi
        nrm = np.linalg.norm(psi)
        logn += 2.0 * np.log(nrm)
        return psi / nrm, logn

    fr = None
    for k, fr in enumerate(ame.frames(inst)):
        if k == 0:
            psi = fr.eig.V[:, 0].astype(complex)
        else:
            t_prev = (k - 1) * dt
            psi, logn = piece(prev, k - 1, 1, t_prev, psi, logn)
            psi, logn = piece(fr, k, 0, t_prev + tau, psi, logn)
        prev = fr
    g0 = fr.eig.V[:, fr.eig.manifolds[0]]
    c = g0.T @ psi
    return float(np.real(np.vdot(c, c))), logn


def trajectory_gradient_fd(inst, jumps_of_traj, baseline: float, delta: float = 1e-5, which=None):
    """Per-trajectory estimate dp/dtheta + (p - b) d log|psi~_T|^2/dtheta by
    central differences of ``replay`` at fixed record. ``jumps_of_traj``: the
    records of one trajectory. Returns (estimate [n_params], p at theta)."""
    which = range(n_params(inst)) if which is None else which
    p0, _ = replay(inst, jumps_of_traj)
    out = np.full(n_params(inst), np.nan)
    for i in which:
        ph, lh = replay(_bumped(inst, i, delta), jumps_of_traj)
        pl, ll = replay(_bumped(inst, i, -delta), jumps_of_traj)
        out[i] = (ph - pl) / (2.0 * delta) + (p0 - baseline) * (lh - ll) / (2.0 * delta)
    return out, p0


def undefined_params(inst) -> np.ndarray:
    """Parameters whose derivative the secular AME does not have at this
    instance: those whose dH_S/dtheta, at a grid point with degenerate levels,
    couples two levels of one degenerate manifold. Moving such a parameter
    lifts the degeneracy, which regroups the Bohr classes of Eq. Lindblad2
    (the generator changes discontinuously). At s = 0 of the transverse-field
    model (B(0) = 0) this is B at the first knot."""
    s_grid, _ = model.grid(inst)
    HX, HZ = model.hamiltonian_terms(inst)
    k = len(inst.sched_s)
    n = inst.n_qubits
    z = model.sigma_z_diagonals(n)
    out = np.zeros(n_params(inst), dtype=bool)
    iu = np.triu_indices(n, k=1)
    for s in s_grid:
        eig = model.eigen_at(inst, float(s), (HX, HZ))
        if eig.nondegenerate:
            continue
        A, B = model.schedule(inst, float(s))
        hat = [float(np.interp(s, inst.sched_s, e)) for e in np.eye(k)]
        dH = [hat[i] * HX for i in range(k)] + [hat[i] * HZ for i in range(k)]
        dH += [B * np.diag(z[i]) for i in range(n)]
        dH += [B * np.diag(z[i] * z[j]) for i, j in zip(*iu)]
        V = eig.V
        for pi, d in enumerate(dH):
            Hp = V.T @ d @ V
            for lev in eig.manifolds:
                if len(lev) > 1:
                    blk = Hp[np.ix_(lev, lev)]
                    if np.max(np.abs(blk - np.diag(np.diag(blk)))) > 1e-9 * max(1.0, np.max(np.abs(Hp))):
                        out[pi] = True
    return out
