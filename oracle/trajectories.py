"""Serial quantum-jump trajectory sampler for the AME (waiting-time algorithm).

Test infrastructure only (see the package docstring).

Sec. IV (simulation procedure) with App. C (waiting times for time-dependent
operators): draw r; propagate the unnormalised state under H_eff until its
squared norm has fallen to r; choose the jump from the probabilities
Pi_i = <A_i^dag A_i> / lambda (App. B.1, Eq. Pi(t)); apply it (Eq. jump),
renormalise, draw a new r and continue.

Readings shared with the CUDA path:
  * the state lives in the computational basis here; the generator is frozen
    on the same symmetric split as the density-matrix oracle (see ``ame``), and
    each frozen piece is propagated with scipy's matrix exponential of
    -i H_eff t, H_eff = V K V^T;
  * the jump time inside a piece is the root of ||exp(-i H_eff t) psi||^2 = r,
    bracketed and solved by Brent's method; a tie (norm equal to r) jumps
    ("refined" timing). With "grid" timing the jump is applied at the end of
    the piece in which the squared norm fell to r, with the state propagated
    through the whole piece (the paper's condition checked at time-step
    resolution only);
  * jump choice with two uniforms (u1, u2). Units (alpha, m, a): qubit alpha,
    source manifold m, target level a, with weight
        w = gamma(E(m) - E(m(a))) |sum_{b in m} M_alpha[a,b] c_b|^2 ,  c = V^T psi .
    Stage one picks (alpha, m) by inverse CDF over alpha ascending, then m
    ascending in energy, with u1; stage two picks a, ascending, with u2. The
    class containing (a, m) is the channel; the sum of its units' weights is
    <A^dag A>, so each channel is drawn with probability Pi_i exactly. The new
    state is A_{alpha,class} psi, normalised;
  * random numbers come from ``philox`` with the stream layout stated there;
  * a jump record names the source and target manifolds by their lowest
    level: inside a degenerate manifold the level that stage two lands on
    depends on the arbitrary eigenbasis, the manifold (hence the channel and
    the new state) does not;
  * truncated model (``inst.n_levels``): the state stays in the span of the
    kept eigenstates; at each grid change it is projected onto the new span
    and rescaled to its norm before the projection, so the weight that leaves
    the kept levels (the leakage) is renormalised away and never counted as
    jump probability (the norm clock is untouched).
"""
from __future__ import annotations

import numpy as np
from scipy import linalg, optimize

from . import ame, lindblad, model, philox


class Piece:
    """No-jump propagation data of one frozen generator."""

    def __init__(self, fr: lindblad.Frame, tau: float):
        self.fr = fr
        V = fr.eig.V
        self.Heff = V @ fr.K @ V.T
        self.U_tau = linalg.expm(-1j * self.Heff * tau)

    def U(self, t: float):
        return linalg.expm(-1j * self.Heff * t)


def choose_jump(fr: lindblad.Frame, psi: np.ndarray, u1: float, u2: float):
    """Stage-one and stage-two draws; returns (alpha, m, a, class id, new psi)."""
    eig = fr.eig
    c = eig.V.T @ psi
    n = fr.M.shape[0]
    nm = len(eig.manifolds)
    lm = eig.level_manifold
    W = np.zeros((n, nm))
    unit_w = {}
    for al in range(n):
        for m, lev in enumerate(eig.manifolds):
            y = fr.M[al][:, lev] @ c[lev]
            w = fr.gam[:, lev[0]] * np.abs(y) ** 2
            unit_w[(al, m)] = w
            W[al, m] = w.sum()
    flat = W.reshape(-1)
    cdf = np.cumsum(flat)
    idx = int(np.searchsorted(cdf, u1 * cdf[-1], side="right"))
    idx = min(idx, len(flat) - 1)
    while flat[idx] <= 0.0 and idx > 0:   # rounding guard: never pick an empty unit
        idx -= 1
    al, m = divmod(idx, nm)
    w = unit_w[(al, m)]
    cdf2 = np.cumsum(w)
    a = int(np.searchsorted(cdf2, u2 * cdf2[-1], side="right"))
    a = min(a, len(w) - 1)
    while w[a] <= 0.0 and a > 0:
        a -= 1
    b0 = eig.manifolds[m][0]
    cls = fr.class_of_pair[a, b0]
    mask = fr.class_of_pair == cls
    A = np.where(mask, fr.R[al], 0.0)
    newc = A @ c
    newc /= np.linalg.norm(newc)
    return al, m, a, cls, eig.V @ newc


class Trajectory:
    def __init__(self, traj: int, seed: int, psi0: np.ndarray):
        self.traj = traj
        self.seed = seed
        self.psi = psi0.astype(complex)
        self.r = philox.first_threshold(seed, traj)
        self.n_jumps = 0
        self.jumps = []

    def project(self, V: np.ndarray) -> float:
        """Project onto the span of V's columns, keeping the norm; returns the
        leaked fraction of the squared norm."""
        n2 = np.vdot(self.psi, self.psi).real
        new = V @ (V.T @ self.psi)
        m2 = np.vdot(new, new).real
        self.psi = new * np.sqrt(n2 / m2)
        return 1.0 - m2 / n2

    def advance(self, piece: Piece, tau: float, t0: float, grid_index: int, half: int, timing: str = "refined"):
        """Propagate through one frozen piece of length tau starting at t0."""
        psi = self.psi
        elapsed = 0.0
        remaining = tau
        while True:
            U = piece.U_tau if elapsed == 0.0 else piece.U(remaining)
            trial = U @ psi
            if np.vdot(trial, trial).real > self.r:
                self.psi = trial
                return
            if timing == "grid":
                tstar = remaining
            else:
                start = psi
                f = lambda t: np.vdot(v := piece.U(t) @ start, v).real - self.r  # noqa: E731
                if f(remaining) > 0.0:   # rounding between the two evaluations
                    self.psi = trial
                    return
                tstar = optimize.brentq(f, 0.0, remaining, xtol=1e-16 * max(tau, 1e-30), rtol=1e-15,
                                        maxiter=200)
            start = psi
            psi = piece.U(tstar) @ start
            psi = psi / np.linalg.norm(psi)
            self.n_jumps += 1
            u1, u2, rnext = philox.jump_draws(self.seed, self.traj, self.n_jumps)
            al, m, a, cls, psi = choose_jump(piece.fr, psi, u1, u2)
            eig = piece.fr.eig
            self.jumps.append(dict(traj=self.traj, grid=grid_index, half=half,
                                   t=t0 + elapsed + tstar, alpha=al,
                                   src=int(eig.manifolds[m][0]),
                                   dst=int(eig.manifolds[eig.level_manifold[a]][0]),
                                   omega=float(eig.E[m] - eig.E[eig.level_manifold[a]])))
            self.r = rnext
            elapsed += tstar
            remaining -= tstar
            if remaining <= 0.0:
                self.psi = psi
                return


def sample(inst, traj_ids, seed=None, timing: str = "refined", return_leak: bool = False):
    """Run the given trajectories over the whole grid (``timing``: "refined" or
    "grid", see the module docstring).

    Returns (p_gs [len(traj_ids), K], jumps (list of dicts), final psi
    [len(traj_ids), N] in the computational basis, normalised), and with
    ``return_leak`` the leaked fraction at each frame change
    [len(traj_ids), K] (zero without truncation).
    """
    seed = inst.seed if seed is None else seed
    s_grid, dt = model.grid(inst)
    tau = 0.5 * dt
    K = len(s_grid)
    p = np.empty((len(traj_ids), K))
    leak = np.zeros((len(traj_ids), K))
    trajs = None
    prev = None
    for k, fr in enumerate(ame.frames(inst)):
        piece = Piece(fr, tau)
        if k == 0:
            psi0 = fr.eig.V[:, 0]
            trajs = [Trajectory(int(t), seed, psi0) for t in traj_ids]
        else:
            t_prev = (k - 1) * dt
            for i, tr in enumerate(trajs):
                tr.advance(prev, tau, t_prev, k - 1, 1, timing)
                if fr.eig.truncated:
                    leak[i, k] = tr.project(fr.eig.V)
                tr.advance(piece, tau, t_prev + tau, k, 0, timing)
        g0 = fr.eig.manifolds[0]
        for i, tr in enumerate(trajs):
            c = fr.eig.V[:, g0].T @ tr.psi
            p[i, k] = float(np.sum(np.abs(c) ** 2) / np.vdot(tr.psi, tr.psi).real)
        prev = piece
    jumps = [j for tr in trajs for j in tr.jumps]
    final = np.array([tr.psi / np.linalg.norm(tr.psi) for tr in trajs])
    if return_leak:
        return p, jumps, final, leak
    return p, jumps, final


def sample_fixed_step(inst, traj_ids, seed=None):
    """The fixed-step unravelling of App. B.1 on the same frozen pieces.

    At the start of each piece (length tau, generator frozen) with normalised
    psi: lambda = sum_i <A_i^dag A_i> = -2 Im <psi|H_eff|psi> (Eq. lambda),
    Delta p = tau lambda, and with a fresh uniform eps a jump happens when
    Delta p > eps; its channel is drawn with the probabilities Pi_i (Eq.
    Pi(t)), and the jump replaces the piece's deterministic evolution. Without
    a jump psi <- exp(-i H_eff tau) psi, renormalised. Piece q (q = 0, 1, ...
    in time order) draws from ``philox.fixed_step_draws(seed, traj, q)``.
    Returns the same triple as ``sample``; jump times are the pieces' starts.
    """
    seed = inst.seed if seed is None else seed
    s_grid, dt = model.grid(inst)
    tau = 0.5 * dt
    K = len(s_grid)
    p = np.empty((len(traj_ids), K))
    psis, jumps, prev = None, [], None

    def step(piece, psi, traj, q, t0, g, half):
        lam = -2.0 * np.vdot(psi, piece.Heff @ psi).imag
        eps, u1, u2 = philox.fixed_step_draws(seed, traj, q)
        if tau * lam > eps:
            al, m, a, cls, new = choose_jump(piece.fr, psi, u1, u2)
            eig = piece.fr.eig
            jumps.append(dict(traj=traj, grid=g, half=half, t=t0, alpha=al, src=int(eig.manifolds[m][0]),
                              dst=int(eig.manifolds[eig.level_manifold[a]][0]),
                              omega=float(eig.E[m] - eig.E[eig.level_manifold[a]])))
            return new
        v = piece.U_tau @ psi
        return v / np.linalg.norm(v)

    for k, fr in enumerate(ame.frames(inst)):
        piece = Piece(fr, tau)
        if k == 0:
            psis = [fr.eig.V[:, 0].astype(complex) for _ in traj_ids]
        else:
            t_prev = (k - 1) * dt
            for i, tr in enumerate(traj_ids):
                psis[i] = step(prev, psis[i], int(tr), 2 * k - 2, t_prev, k - 1, 1)
                if fr.eig.truncated:  # frame change onto the kept levels, renormalised
                    v = fr.eig.V @ (fr.eig.V.T @ psis[i])
                    psis[i] = v / np.linalg.norm(v)
                psis[i] = step(piece, psis[i], int(tr), 2 * k - 1, t_prev + tau, k, 0)
        g0 = fr.eig.manifolds[0]
        for i in range(len(traj_ids)):
            c = fr.eig.V[:, g0].T @ psis[i]
            p[i, k] = float(np.sum(np.abs(c) ** 2))
        prev = piece
    return p, jumps, np.array(psis)

