"""Density-matrix solution of the AME on the shared time grid.

Test infrastructure only (see the package docstring).

Time discretisation (a reading: the paper leaves the integrator open, Sec. IV):
the generator is frozen at s_{k-1} for the first half of [t_{k-1}, t_k] and at
s_k for the second half (a symmetric split of the time-dependent generator).
Each frozen half-step is integrated exactly (Taylor series of exp(L tau) to
machine precision, or the closed form for generic spectra). The quantum-jump
trajectories of Sec. IV, taken on the same split, average to exactly this
density matrix (App. B.2); this is the "split-exact" AME.

The state starts in the ground state of H_S(0) (Sec. V.A). Observable: the
population of the lowest degenerate manifold of H_S(s_k), recorded after the
second half-step into s_k.
"""
from __future__ import annotations

import numpy as np

from . import lindblad, model


def spectral_bound(inst) -> float:
    """Upper bound on twice the spectral radius of H_S(s) over the schedule:
    the range of any Bohr frequency."""
    n = inst.n_qubits
    hz_sum = float(np.sum(np.abs(inst.hz)))
    j_sum = float(np.sum(np.abs(np.triu(inst.J, 1))))
    r = max(abs(a) * n + abs(b) * (hz_sum + j_sum) for a, b in zip(inst.sched_A, inst.sched_B))
    return 2.0 * r * 1.01 + 1.0


def frames(inst):
    """The generator at every grid point (an iterator, to bound memory)."""
    terms = model.hamiltonian_terms(inst)
    z = model.sigma_z_diagonals(inst.n_qubits)
    wmax = spectral_bound(inst)
    s_grid, _ = model.grid(inst)
    for s in s_grid:
        yield lindblad.Frame(inst, float(s), terms=terms, zdiag=z, wmax=wmax)


def half_step(fr: lindblad.Frame, rho: np.ndarray, tau: float, closed_form: bool) -> np.ndarray:
    if closed_form and fr.generic:
        return fr.propagate_generic(rho, tau)
    return fr.propagate(rho, tau)


def run(inst, closed_form: bool = True, keep_states: bool = False):
    """Split-exact AME over the grid.

    Returns a dict with ``s`` (grid), ``p_gs`` (ground-manifold population at
    each grid point), ``rho_final`` (eigenframe of s = 1) and, optionally,
    ``states`` (every rho in its own eigenframe).
    """
    s_grid, dt = model.grid(inst)
    tau = 0.5 * dt
    p_gs = np.empty(len(s_grid))
    states = [] if keep_states else None
    prev = None
    rho = None
    for k, fr in enumerate(frames(inst)):
        if k == 0:
            rho = np.zeros((fr.N, fr.N), dtype=complex)
            rho[0, 0] = 1.0
        else:
            rho = half_step(prev, rho, tau, closed_form)           # frozen at s_{k-1}
            O = fr.eig.V.T @ prev.eig.V                          # frame s_{k-1} -> s_k
            rho = O @ rho @ O.T
            rho = half_step(fr, rho, tau, closed_form)             # frozen at s_k
        g0 = fr.eig.manifolds[0]
        p_gs[k] = float(np.real(np.trace(rho[np.ix_(g0, g0)])))
        if keep_states:
            states.append(rho.copy())
        prev = fr
    out = {"s": s_grid, "p_gs": p_gs, "rho_final": rho}
    if keep_states:
        out["states"] = states
    return out
