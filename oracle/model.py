"""TFIM system Hamiltonian, schedule and instantaneous eigenstructure.

Test infrastructure only (see the package docstring).

Sec. V, Eq. H_S: H_S(s) = A(s) H^X + B(s) H^Z with H^X = -sum_i sx_i and (in the
explicit-sign form used by this library) H^Z = sum_i hz_i sz_i + sum_{i<j} J_ij sz_i sz_j.
Basis: index x = sum_i bit_i 2^i, qubit i <-> bit i, bit 0 <-> sz = +1.

Sec. II, Eq. Lindblad2: the Lindblad operators are built from the instantaneous
eigenstates and group level pairs by equal Bohr frequency. Readings (the paper
states exact equality only):
  * levels are sorted ascending; consecutive eigenvalues closer than
    tol = 1e-12 * max(1, max|eps|) form one degenerate manifold, whose energy is
    the mean of its eigenvalues;
  * the Bohr frequency of a level pair (a, b) is E(m(b)) - E(m(a)); pairs in the
    same manifold have omega = 0;
  * Bohr frequencies of distinct manifold pairs are sorted and chained where
    consecutive values differ by at most tol; a chain wider than tol is an
    ambiguous grouping and is rejected.
"""
from __future__ import annotations

import numpy as np

SX = np.array([[0.0, 1.0], [1.0, 0.0]])
SZ = np.array([[1.0, 0.0], [0.0, -1.0]])


def op_on(qubit: int, op: np.ndarray, n: int) -> np.ndarray:
    """Dense operator acting as ``op`` on ``qubit`` and identity elsewhere.
    np.kron puts its first factor on the most significant index bits, so the
    factors run from qubit n-1 down to qubit 0."""
    out = np.array([[1.0]])
    for q in range(n - 1, -1, -1):
        out = np.kron(out, op if q == qubit else np.eye(2))
    return out


def hamiltonian_terms(inst):
    """(H^X, H^Z) as dense real matrices (Sec. V, Eq. H_S)."""
    n = inst.n_qubits
    HX = -sum(op_on(i, SX, n) for i in range(n))
    HZ = sum(inst.hz[i] * op_on(i, SZ, n) for i in range(n))
    for i in range(n):
        for j in range(i + 1, n):
            if inst.J[i, j] != 0.0:
                HZ = HZ + inst.J[i, j] * (op_on(i, SZ, n) @ op_on(j, SZ, n))
    return HX, HZ


def sigma_z_diagonals(n: int) -> np.ndarray:
    """(n, 2^n) diagonals of sz_alpha, the system-bath coupling operators A_alpha
    (Sec. V, Eq. SBm: independent sz coupling per qubit)."""
    return np.array([np.diag(op_on(a, SZ, n)) for a in range(n)])


def schedule(inst, s: float):
    """Piecewise-linear A(s), B(s) through the instance's knots."""
    return (float(np.interp(s, inst.sched_s, inst.sched_A)),
            float(np.interp(s, inst.sched_s, inst.sched_B)))


def grid(inst):
    """s_k = k / (K - 1), k = 0..K-1, and the time step dt = t_f / (K - 1)."""
    K = inst.n_grid
    return np.arange(K) / (K - 1), inst.t_f / (K - 1)


def energy_tol(evals: np.ndarray) -> float:
    return 1e-12 * max(1.0, float(np.max(np.abs(evals))))


class Eigen:
    """Instantaneous eigensystem of H_S(s) with its degenerate manifolds.

    keep > 0 keeps only the lowest ``keep`` levels (a truncated model: the
    system's Hilbert space is the span of those eigenstates at every s). The
    cut must fall between manifolds: a level just above the cut within the
    tolerance of the level just below it raises ValueError. The tolerance is
    that of the kept levels."""

    def __init__(self, H: np.ndarray, keep: int = 0):
        evals, V = np.linalg.eigh(H)
        if 0 < keep < len(evals):
            if evals[keep] - evals[keep - 1] <= energy_tol(evals[:keep]):
                raise ValueError(f"keeping {keep} levels splits a degenerate manifold")
            evals, V = evals[:keep], V[:, :keep]
        self.evals = evals
        self.V = V
        self.truncated = V.shape[0] != V.shape[1]
        self.tol = energy_tol(evals)
        groups = [[0]]
        for a in range(1, len(evals)):
            if evals[a] - evals[a - 1] <= self.tol:
                groups[-1].append(a)
            else:
                groups.append([a])
        self.manifolds = [np.array(g) for g in groups]
        self.E = np.array([evals[g].mean() for g in self.manifolds])
        self.level_manifold = np.empty(len(evals), dtype=int)
        for m, g in enumerate(self.manifolds):
            self.level_manifold[g] = m
        # Bohr frequency of level pair (b -> a): omega[a, b] = E(m(b)) - E(m(a)).
        El = self.E[self.level_manifold]
        self.omega = El[None, :] - El[:, None]

    @property
    def nondegenerate(self) -> bool:
        return len(self.manifolds) == len(self.evals)


def eigen_at(inst, s: float, terms=None) -> Eigen:
    """Eigensystem of H_S(s), truncated to inst.n_levels levels when set."""
    HX, HZ = terms if terms is not None else hamiltonian_terms(inst)
    A, B = schedule(inst, s)
    return Eigen(A * HX + B * HZ, keep=getattr(inst, "n_levels", 0))


def bohr_classes(eig: Eigen):
    """Group the manifold pairs (ma, mb), ma != mb, into classes of equal Bohr
    frequency omega = E(mb) - E(ma) (Sec. II, Eq. Lindblad2).

    Returns a list of (omega, [(ma, mb), ...]); the omega = 0 class, made of all
    (m, m) pairs, comes first; the others follow in increasing omega.
    """
    nm = len(eig.E)
    ma, mb = np.meshgrid(np.arange(nm), np.arange(nm), indexing="ij")
    off = ma != mb
    ma, mb = ma[off], mb[off]
    w = eig.E[mb] - eig.E[ma]
    order = np.argsort(w, kind="stable")
    w, ma, mb = w[order], ma[order], mb[order]
    classes = [(0.0, [(m, m) for m in range(nm)])]
    if len(w) == 0:
        return classes
    # chains: consecutive sorted frequencies no farther apart than tol
    brk = np.flatnonzero(np.diff(w) > eig.tol) + 1
    starts = np.r_[0, brk]
    ends = np.r_[brk, len(w)]
    if np.any(w[ends - 1] - w[starts] > eig.tol):
        raise ValueError("ambiguous Bohr-frequency grouping: chain wider than tolerance")
    means = np.add.reduceat(w, starts) / (ends - starts)
    mal, mbl = ma.tolist(), mb.tolist()
    for ci, (st, en) in enumerate(zip(starts.tolist(), ends.tolist())):
        classes.append((float(means[ci]), list(zip(mal[st:en], mbl[st:en]))))
    return classes
