"""Pins of the gradient oracle (oracle/gradient.py) to facts outside it: a
closed form differentiated symbolically, an exact scaling identity of the
Hamiltonian family, and the statistical identity between the trajectory
estimate and the derivative of the density matrix."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import gradient as G
from oracle import trajectories


def two_point_instance(A0, A1, B0, B1, h, eta_g2=0.0):
    """One qubit, two schedule knots and a two-point grid: the state starts in
    the ground state of H(0) = -A0 sx + B0 h sz, turns a phase for a
    half-step, is taken into the eigenframe of H(1) and turns phases again.
    Without a bath its final ground-state population is the squared overlap of
    the two ground states."""
    return W.Instance(n_qubits=1, hz=np.array([h]), J=np.zeros((1, 1)), sched_s=np.array([0.0, 1.0]),
                      sched_A=np.array([A0, A1]), sched_B=np.array([B0, B1]), eta_g2=eta_g2, t_f=0.7,
                      n_grid=2, lamb_shift=False, seed=3)


def test_two_point_gradient_closed_form():
    sympy = pytest.importorskip("sympy")
    a0, a1, b0, b1, h = sympy.symbols("a0 a1 b0 b1 h", real=True)
    # ground state of -a sx + c sz has Bloch vector (a, 0, -c) / sqrt(a^2 + c^2);
    # the squared overlap of two states is (1 + n0 . n1) / 2
    r0 = sympy.sqrt(a0 ** 2 + (b0 * h) ** 2)
    r1 = sympy.sqrt(a1 ** 2 + (b1 * h) ** 2)
    P = (1 + (a0 * a1 + b0 * b1 * h ** 2) / (r0 * r1)) / 2
    vals = {a0: 5.0, a1: 1.3, b0: 0.4, b1: 4.2, h: -0.7}
    ref = [float(sympy.diff(P, v).subs(vals)) for v in (a0, a1, b0, b1, h)]
    inst = two_point_instance(*[vals[v] for v in (a0, a1, b0, b1, h)])
    fd = G.ame_gradient_fd(inst, delta=1e-5)
    np.testing.assert_allclose(fd, ref, rtol=1e-7, atol=1e-9)
    # no bath: no jumps, the record is empty and the estimate is dp/dtheta
    est, p0 = G.trajectory_gradient_fd(inst, [], baseline=0.3)
    assert abs(p0 - float(P.subs(vals))) < 1e-12
    np.testing.assert_allclose(est, ref, rtol=1e-7, atol=1e-9)


def hot_instance(seed=3):
    return W.tfim_instance(2, seed, eta_g2=0.05, t_f=4.0, n_grid=10, seed=7)


def test_field_scaling_identity():
    """H^Z is linear in (hz, J), so scaling them all by lambda is scaling B(s)
    at every knot by lambda: sum hz dP/dhz + sum J dP/dJ = sum_k B_k dP/dB_k,
    for the density matrix and for every trajectory's record-fixed estimate."""
    inst = hot_instance()
    th = G.param_vector(inst)
    k = len(inst.sched_s)
    fd = G.ame_gradient_fd(inst, delta=1e-4)
    lhs = np.dot(th[2 * k:], fd[2 * k:])
    rhs = np.dot(th[k:2 * k], np.nan_to_num(fd[k:2 * k]))
    assert abs(lhs - rhs) < 1e-7 * max(1.0, abs(lhs)), (lhs, rhs)
    p, jumps, _ = trajectories.sample(inst, list(range(6)))
    assert len(jumps) > 0
    for t in range(6):
        est, _ = G.trajectory_gradient_fd(inst, [j for j in jumps if j["traj"] == t], baseline=0.5)
        lhs = np.dot(th[2 * k:], est[2 * k:])
        rhs = np.dot(th[k:2 * k], est[k:2 * k])
        assert abs(lhs - rhs) < 1e-7 * max(1.0, abs(lhs)), (t, lhs, rhs)


def test_first_knot_of_B_is_undefined_at_degenerate_start():
    inst = hot_instance()
    und = G.undefined_params(inst)
    k = len(inst.sched_s)
    assert und[k] and und.sum() == 1  # B at s = 0 only (H(0) = -A sum sx is degenerate for n = 2)


@pytest.mark.slow
def test_trajectory_estimate_is_unbiased():
    """Mean of the record-fixed estimates over sampled trajectories against the
    central differences of the density matrix (hot bath, two qubits): within
    4 sigma of the sample mean for every parameter."""
    inst = hot_instance()
    M = 240
    p, jumps, _ = trajectories.sample(inst, list(range(M)))
    b = float(p[:, -1].mean())
    by = {t: [] for t in range(M)}
    for j in jumps:
        by[j["traj"]].append(j)
    est = np.array([G.trajectory_gradient_fd(inst, by[t], baseline=b)[0] for t in range(M)])
    fd = G.ame_gradient_fd(inst, delta=1e-4)
    m, se = est.mean(axis=0), est.std(axis=0, ddof=1) / math.sqrt(M)
    z = np.abs(m - fd) / np.maximum(se, 1e-12)
    assert np.all(z < 4.0), (m, fd, se)
    # the estimates are not trivially small: the bath moves the population
    assert np.max(np.abs(fd)) > 0.1
