"""Seeded synthetic inputs for the adiabatic-master-equation trajectory path.

This module is shared by the oracle, the tests and the benchmark. It holds
no arithmetic of the method itself: it only draws Ising coefficients from a
seed, writes down schedule knots and bath constants, and converts physical
units. Everything is in angular units with hbar = 1: energies and rates in
rad/ns, times in ns, inverse temperature beta in ns.

Instance family (transverse-field Ising annealing, Sec. V, Eq. H_S):
    H(s) = A(s) * (-sum_i sx_i) + B(s) * (sum_i hz_i sz_i + sum_{i<j} J_ij sz_i sz_j)
with a linear schedule A(s) = 2*pi*(1-s), B(s) = 2*pi*s, and h_i, J_ij drawn
as sign * magnitude, sign uniform in {-1, +1}, magnitude uniform in [0.1, 1],
on the complete graph. The paper's own convention H^Z = -sum h sz + sum J sz sz
(Sec. V) maps to hz = -h; the synthetic family uses hz = h directly.

Bath (Sec. V, Ohmic spectral density): eta*g^2 = 1e-3, omega_c = 8*pi rad/ns,
T = 12.1 mK, independent sz coupling per qubit.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Physical constants (CODATA 2018, exact SI values for kB and h).
KB_J_PER_K = 1.380649e-23
HBAR_J_S = 1.054571817e-34


def beta_from_mk(t_mk: float) -> float:
    """Inverse temperature in ns for a temperature given in mK (hbar = 1,
    angular units): beta = hbar / (kB T)."""
    omega_t = KB_J_PER_K * (t_mk * 1e-3) / HBAR_J_S  # rad/s
    return 1.0 / (omega_t * 1e-9)  # ns


@dataclasses.dataclass
class Instance:
    """One annealing problem: Ising terms, schedule knots, bath and grid."""
    n_qubits: int
    hz: np.ndarray            # (n,) rad/ns before the schedule factor
    J: np.ndarray             # (n, n) upper triangle used, i < j
    sched_s: np.ndarray       # knots of the piecewise-linear schedule
    sched_A: np.ndarray       # A(s) at the knots, rad/ns
    sched_B: np.ndarray       # B(s) at the knots, rad/ns
    eta_g2: float = 1e-3
    omega_c: float = 8.0 * math.pi
    beta: float = dataclasses.field(default_factory=lambda: beta_from_mk(12.1))
    lamb_shift: bool = True
    t_f: float = 10.0         # ns
    n_grid: int = 1000
    M: int = 1000             # trajectories
    seed: int = 1             # trajectory random-stream seed
    n_levels: int = 0         # keep the lowest n_levels instantaneous eigenstates (0: all)

    @property
    def N(self) -> int:
        return 1 << self.n_qubits


def linear_schedule():
    """A(s) = 2*pi*(1-s), B(s) = 2*pi*s (units 2*pi GHz -> rad/ns)."""
    two_pi = 2.0 * math.pi
    return (np.array([0.0, 1.0]), np.array([two_pi, 0.0]), np.array([0.0, two_pi]))


def random_ising(n_qubits: int, seed: int, discrete: bool = False):
    """Seeded h_i, J_ij = sign * magnitude on the complete graph.

    magnitude ~ U[0.1, 1] (continuous), or uniform over {0.1, 0.2, ..., 1.0}
    when ``discrete`` is set; sign ~ U{-1, +1}.
    """
    rng = np.random.Generator(np.random.Philox(seed))

    def draw(size):
        sign = rng.choice(np.array([-1.0, 1.0]), size=size)
        if discrete:
            mag = rng.integers(1, 11, size=size) / 10.0
        else:
            mag = rng.uniform(0.1, 1.0, size=size)
        return sign * mag

    hz = draw(n_qubits)
    J = np.zeros((n_qubits, n_qubits))
    iu = np.triu_indices(n_qubits, k=1)
    J[iu] = draw(len(iu[0]))
    return hz, J


def tfim_instance(n_qubits: int, instance_seed: int, **kw) -> Instance:
    """Random complete-graph TFIM drawn from ``instance_seed``; keyword
    arguments set the remaining Instance fields (including the trajectory
    stream ``seed``)."""
    hz, J = random_ising(n_qubits, instance_seed)
    s, A, B = linear_schedule()
    return Instance(n_qubits=n_qubits, hz=hz, J=J, sched_s=s, sched_A=A, sched_B=B, **kw)


def cfg_small(**kw) -> Instance:
    """4 qubits (N = 16, all levels), t_f = 10 ns, 1000-point grid, M = 1000."""
    base = dict(t_f=10.0, n_grid=1000, M=1000, seed=1710_03431)
    base.update(kw)
    return tfim_instance(4, 1710_03431, **base)


def cfg_main(t_f: float = 10.0, **kw) -> Instance:
    """8 qubits (N = 256, all levels), t_f in {10, 100} ns, 2000-point grid,
    M = 10^4 trajectories."""
    base = dict(t_f=t_f, n_grid=2000, M=10_000, seed=1710_03432)
    base.update(kw)
    return tfim_instance(8, 1710_03432, **base)


def chain8_instance(**kw) -> Instance:
    """The 8-qubit ferromagnetic chain of Sec. V.A (Eq. Ising): h_1 = 1/4,
    other h = 0, J_{i,i+1} = -1 (seven bonds), in the paper's sign convention
    (hz = -h), with the linear schedule (the D-Wave schedule is only given as
    a figure)."""
    n = 8
    hz = np.zeros(n)
    hz[0] = -0.25
    J = np.zeros((n, n))
    for i in range(n - 1):
        J[i, i + 1] = -1.0
    s, A, B = linear_schedule()
    return Instance(n_qubits=n, hz=hz, J=J, sched_s=s, sched_A=A, sched_B=B, **kw)


def case0989_instance(**kw) -> Instance:
    """The 8-qubit small-gap instance of Sec. V.B (Eq. Case0989), paper sign
    convention (hz = -h), linear schedule."""
    h = np.array([-2, -2, 2, -3, 1, 3, -3, 3], dtype=float) / 3.0
    Jv = {(0, 4): 1, (0, 5): -3, (0, 6): -1, (0, 7): -1,
          (1, 4): -1, (1, 5): -2, (1, 6): 2, (1, 7): -3,
          (2, 4): -2, (2, 5): -1, (2, 6): -3, (2, 7): -2,
          (3, 4): -3, (3, 5): -3, (3, 6): -1, (3, 7): -3}
    J = np.zeros((8, 8))
    for (i, j), v in Jv.items():
        J[i, j] = v / 3.0
    s, A, B = linear_schedule()
    return Instance(n_qubits=8, hz=-h, J=J, sched_s=s, sched_A=A, sched_B=B, **kw)


def cfg_batch(n_instances: int = 64, qubits=(6, 7, 8), M: int = 2048, n_grid: int = 1000, t_f: float = 20.0,
              **kw):
    """Batch of independent instances of uneven size: instance i has
    qubits[i % len(qubits)] qubits and its own seeded couplings (instance seed
    1710_03500 + i) and trajectory streams, t_f = 20 ns, 1000-point grid,
    M = 2048 trajectories each."""
    out = []
    for i in range(n_instances):
        n = qubits[i % len(qubits)]
        base = dict(t_f=t_f, n_grid=n_grid, M=M, seed=1710_03500 + 7919 * i)
        base.update(kw)
        out.append(tfim_instance(n, 1710_03500 + i, **base))
    return out



def cfg_grad(n_knots: int = 8, **kw) -> Instance:
    """Differentiation workload: the 8-qubit complete-graph instance of
    ``cfg_main`` (N = 256) with its linear schedule written as n_knots
    piecewise-linear control points s_k = k / (n_knots - 1) of A and B, t_f =
    10 ns, 2000-point grid, M = 2^14 trajectories. Parameters: the 2 n_knots
    control values, the 8 fields and the 28 couplings."""
    base = dict(t_f=10.0, n_grid=2000, M=1 << 14, seed=1710_03433)
    base.update(kw)
    inst = tfim_instance(8, 1710_03432, **base)
    s = np.linspace(0.0, 1.0, n_knots)
    inst.sched_s = s
    inst.sched_A = 2.0 * math.pi * (1.0 - s)
    inst.sched_B = 2.0 * math.pi * s
    return inst
