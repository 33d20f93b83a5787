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

Truncated model (``inst.n_levels``: the lowest levels only, a reading of the
paper's 16-qubit use; the paper does not discuss truncation): the frame
change O = V_k^T V_{k-1} is then not orthogonal; the weight it moves out of
the kept levels (the leakage, 1 - tr(O rho O^T)) is recorded and renormalised
away, never counted as jump probability.

``run_continuous`` integrates the same AME without the grid (Sec. II, Eqs.
ME2-H, ME2-L): the generator is rebuilt from the eigensystem of H_S(s(t)) at
every time the adaptive integrator asks for (Dormand-Prince 8(5,3)), which
bounds the discretisation error of the grid.
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
    leak = np.zeros(len(s_grid))
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
            tr0 = np.trace(rho).real
            rho = O @ rho @ O.T
            if fr.eig.truncated:
                tr1 = np.trace(rho).real
                leak[k] = 1.0 - tr1 / tr0
                rho = rho * (tr0 / tr1)
            rho = half_step(fr, rho, tau, closed_form)             # frozen at s_k
        g0 = fr.eig.manifolds[0]
        p_gs[k] = float(np.real(np.trace(rho[np.ix_(g0, g0)])))
        if keep_states:
            states.append(rho.copy())
        prev = fr
    out = {"s": s_grid, "p_gs": p_gs, "rho_final": rho, "leak": leak}
    if keep_states:
        out["states"] = states
    return out


def run_continuous(inst, rtol: float = 1e-10, atol: float = 1e-12):
    """The AME with the generator of the instantaneous s(t) = t / t_f at every
    stage of an adaptive Dormand-Prince 8(5,3) integration (scipy DOP853) of
    d rho / dt = L_{s(t)}[rho] in the computational basis; the generator acts
    in the eigenframe of H_S(s(t)) as in ``lindblad.Frame``. Returns ``s`` (the
    grid) and ``p_gs`` (ground-manifold population of H_S(s_k) at each grid
    point), comparable with ``run``."""
    from scipy.integrate import solve_ivp

    terms = model.hamiltonian_terms(inst)
    z = model.sigma_z_diagonals(inst.n_qubits)
    wmax = spectral_bound(inst)
    s_grid, _ = model.grid(inst)
    t_grid = s_grid * inst.t_f
    N = inst.N

    def rhs(t, y):
        s = min(max(t / inst.t_f, 0.0), 1.0)
        fr = lindblad.Frame(inst, s, terms=terms, zdiag=z, wmax=wmax)
        rho = (y[: N * N] + 1j * y[N * N:]).reshape(N, N)
        V = fr.eig.V
        d = V @ fr.apply(V.T @ rho @ V) @ V.T
        return np.concatenate([d.real.reshape(-1), d.imag.reshape(-1)])

    eig0 = model.eigen_at(inst, 0.0, terms)
    psi0 = eig0.V[:, 0]
    rho0 = np.outer(psi0, psi0).astype(complex)
    y0 = np.concatenate([rho0.real.reshape(-1), rho0.imag.reshape(-1)])
    sol = solve_ivp(rhs, (0.0, inst.t_f), y0, method="DOP853", t_eval=t_grid, rtol=rtol, atol=atol)
    if not sol.success:
        raise RuntimeError("continuous AME integration failed: " + sol.message)
    p_gs = np.empty(len(s_grid))
    for k, s in enumerate(s_grid):
        eig = model.eigen_at(inst, float(s), terms)
        rho = (sol.y[: N * N, k] + 1j * sol.y[N * N:, k]).reshape(N, N)
        g0 = eig.V[:, eig.manifolds[0]]
        p_gs[k] = float(np.real(np.trace(g0.T @ rho @ g0)))
    return {"s": s_grid, "p_gs": p_gs, "rho_final": (sol.y[: N * N, -1] + 1j * sol.y[N * N:, -1]).reshape(N, N)}
