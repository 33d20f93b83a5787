"""Pins that tie the FP64 oracle to facts outside itself: library routines it
does not use, closed forms, invariants of the Lindblad generator, brute force
on tiny systems and statistical laws of the jump process."""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats
from scipy.linalg import expm

import workloads as W
from oracle import ame, bath, lindblad, model, philox, trajectories

ETA, WC = 1e-3, 8.0 * math.pi
BETA = W.beta_from_mk(12.1)


# --- Philox4x64-10 (SC'11) against numpy's independent implementation ---------
@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (1, 0, 0, 0)),
    ((1, 2), (1, 0, 0, 0)),
    ((0xDEADBEEF12345678, philox.KEY_HI), (17, 3, 0, 0)),
    ((2**64 - 1, 2**63 + 5), (2**64 - 1, 2**64 - 1, 7, 9)),
])
def test_philox_known_answer_vs_numpy(key, ctr):
    # numpy increments its 256-bit counter before each block.
    c = sum(int(v) << (64 * i) for i, v in enumerate(ctr)) - 1
    prev = [(c >> (64 * i)) & philox.MASK64 for i in range(4)]
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
    assert tuple(int(x) for x in g.random_raw(4)) == philox.philox4x64(ctr, key)


def test_uniform_open_interval():
    assert 0.0 < philox.uniform(0) < 1e-15
    assert 1.0 - 1e-15 < philox.uniform(2**64 - 1) < 1.0


# --- Ohmic bath -----------------------------------------------------------------
def test_gamma_kms_and_limit():
    w = np.linspace(0.01, 80.0, 200)
    g_pos = bath.gamma(w, ETA, WC, BETA)
    g_neg = bath.gamma(-w, ETA, WC, BETA)
    np.testing.assert_allclose(g_neg, np.exp(-BETA * w) * g_pos, rtol=1e-12)   # Eq. KMS
    assert abs(bath.gamma(1e-9, ETA, WC, BETA) - bath.gamma(0.0, ETA, WC, BETA)) < 1e-11
    assert np.all(g_pos > 0) and np.all(g_neg > 0)


@pytest.mark.parametrize("w", [-40.0, -3.0, -0.2, 0.0, 0.7, 6.0, 55.0, 180.0])
def test_lamb_shift_zero_temperature_closed_form(w):
    # T -> 0: gamma = 2 pi eta g^2 w e^{-w/wc} for w > 0, else 0, and
    # S(w) = eta g^2 [-wc + w e^{-w/wc} Ei(w/wc)].
    ref = ETA * (-WC + (w * math.exp(-w / WC) * special.expi(w / WC) if w != 0 else 0.0))
    assert abs(bath.lamb_shift_direct(w, ETA, WC, 1e7) - ref) < 1e-12


def test_lamb_shift_table_matches_quadrature():
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(-150, 150, 12), rng.uniform(-2, 2, 6), [0.0]])
    got = bath.lamb_shift(xs, ETA, WC, BETA, wmax=150.0)
    ref = np.array([bath.lamb_shift_direct(x, ETA, WC, BETA) for x in xs])
    assert np.max(np.abs(got - ref)) < 2e-8


def test_lamb_shift_is_principal_value_of_gamma():
    # Independent route: S(w) = (1/2pi) int_0^inf [g(w-x) - g(w+x)] / x dx.
    w = 3.3
    f = lambda x: (bath.gamma(w - x, ETA, WC, BETA) - bath.gamma(w + x, ETA, WC, BETA)) / x  # noqa: E731
    v = sum(integrate.quad(f, lo, hi, limit=300, epsabs=1e-15)[0]
            for lo, hi in [(1e-300, 1.0), (1.0, 30.0), (30.0, 2000.0)])
    assert abs(v / (2 * math.pi) - bath.lamb_shift_direct(w, ETA, WC, BETA)) < 1e-11


# --- Hamiltonian --------------------------------------------------------------------
def _classical_energy(inst, x):
    z = [1 - 2 * ((x >> i) & 1) for i in range(inst.n_qubits)]
    e = sum(inst.hz[i] * z[i] for i in range(inst.n_qubits))
    for i in range(inst.n_qubits):
        for j in range(i + 1, inst.n_qubits):
            e += inst.J[i, j] * z[i] * z[j]
    return e


def test_hamiltonian_against_brute_force():
    inst = W.tfim_instance(3, 11)
    HX, HZ = model.hamiltonian_terms(inst)
    for x in range(8):
        assert abs(HZ[x, x] - _classical_energy(inst, x)) < 1e-13
        for y in range(8):
            flips = bin(x ^ y).count("1")
            assert HX[x, y] == (-1.0 if flips == 1 else 0.0)
    assert np.allclose(HZ, np.diag(np.diag(HZ)))


def test_single_qubit_spectrum_and_s0_multiplicities():
    inst = W.tfim_instance(1, 2)
    for s in [0.0, 0.3, 0.8, 1.0]:
        A, B = model.schedule(inst, s)
        e = model.eigen_at(inst, s).evals
        r = math.hypot(A, B * inst.hz[0])
        np.testing.assert_allclose(e, [-r, r], atol=1e-13)
    inst = W.tfim_instance(4, 3)
    eig = model.eigen_at(inst, 0.0)
    assert [len(m) for m in eig.manifolds] == [1, 4, 6, 4, 1]
    np.testing.assert_allclose(eig.E, -2 * math.pi * np.array([4, 2, 0, -2, -4]), atol=1e-12)


# --- Generator invariants ------------------------------------------------------------
def _rand_rho(N, seed):
    g = np.random.default_rng(seed)
    X = g.normal(size=(N, N)) + 1j * g.normal(size=(N, N))
    r = X @ X.conj().T
    return r / np.trace(r)


@pytest.mark.parametrize("s", [0.0, 0.37, 1.0])
def test_generator_taylor_vs_dense_superoperator(s):
    inst = W.tfim_instance(2, 5)
    fr = lindblad.Frame(inst, s)
    rho = _rand_rho(4, 1)
    a = fr.propagate(rho, 0.4)
    b = (expm(fr.superoperator() * 0.4) @ rho.reshape(-1)).reshape(4, 4)
    assert np.max(np.abs(a - b)) < 1e-13


def test_generic_closed_form_vs_taylor():
    inst = W.tfim_instance(3, 7)
    fr = lindblad.Frame(inst, 0.55)
    assert fr.generic
    rho = _rand_rho(8, 2)
    assert np.max(np.abs(fr.propagate(rho, 0.25) - fr.propagate_generic(rho, 0.25))) < 1e-13


@pytest.mark.parametrize("s", [0.0, 0.5])
def test_trace_hermiticity_positivity(s):
    inst = W.tfim_instance(3, 8, eta_g2=0.05)
    fr = lindblad.Frame(inst, s)
    rho = _rand_rho(8, 3)
    d = fr.apply(rho)
    assert abs(np.trace(d)) < 1e-12
    assert np.max(np.abs(d - d.conj().T)) < 1e-12
    r2 = fr.propagate(rho, 1.0)
    assert abs(np.trace(r2) - 1) < 1e-12
    assert np.min(np.linalg.eigvalsh(0.5 * (r2 + r2.conj().T))) > -1e-12


def test_gibbs_state_is_fixed_point():
    # KMS detailed balance (Eq. KMS): the frozen-s dissipator annihilates exp(-beta H_S).
    inst = W.tfim_instance(3, 9, eta_g2=0.02)
    fr = lindblad.Frame(inst, 0.62)
    p = np.exp(-inst.beta * (fr.eig.evals - fr.eig.evals[0]))
    rho = np.diag(p / p.sum()).astype(complex)
    assert np.max(np.abs(fr.apply(rho))) < 1e-14


def test_decay_rates_are_contractive_and_s0_blocks_scalar():
    inst = W.tfim_instance(4, 10)
    for s in [0.0, 0.2, 0.9]:
        fr = lindblad.Frame(inst, s)
        assert np.all(np.diag(fr.K).imag <= 1e-15)   # ||exp(-i K t)|| <= 1 (App. A)
    fr = lindblad.Frame(inst, 0.0)
    for m in fr.eig.manifolds:
        blk = fr.K[np.ix_(m, m)]
        assert np.max(np.abs(blk - blk[0, 0] * np.eye(len(m)))) < 1e-12


def test_relaxation_rate_formula():
    # Eq. inctunnrate: lambda_{1->0} = sum_alpha gamma(w_10) |<0|sz_alpha|1>|^2.
    inst = W.tfim_instance(3, 12)
    fr = lindblad.Frame(inst, 0.45)
    V = fr.eig.V
    w10 = fr.eig.evals[1] - fr.eig.evals[0]
    lam = sum(bath.gamma(w10, inst.eta_g2, inst.omega_c, inst.beta) *
              (V[:, 0] @ model.op_on(a, model.SZ, 3) @ V[:, 1]) ** 2 for a in range(3))
    assert abs(lam - np.sum(fr.R[:, 0, 1] ** 2)) < 1e-15


def test_degenerate_generator_is_basis_independent():
    inst = W.tfim_instance(3, 13)
    fr = lindblad.Frame(inst, 0.0)
    rho = _rand_rho(8, 4)
    V = fr.eig.V
    a = V @ fr.propagate(V.T @ rho @ V, 0.3) @ V.T
    g = np.random.default_rng(5)
    for m in fr.eig.manifolds:           # rotate each manifold by a random orthogonal matrix
        Q, _ = np.linalg.qr(g.normal(size=(len(m), len(m))))
        fr.eig.V[:, m] = fr.eig.V[:, m] @ Q
    fr3 = _frame_with_basis(inst, 0.0, fr.eig.V)
    b = fr.eig.V @ fr3.propagate(fr.eig.V.T @ rho @ fr.eig.V, 0.3) @ fr.eig.V.T
    assert np.max(np.abs(a - b)) < 1e-13


def _frame_with_basis(inst, s, V):
    orig = np.linalg.eigh

    def fake(H):
        e, _ = orig(H)
        return e, V
    np.linalg.eigh = fake
    try:
        return lindblad.Frame(inst, s)
    finally:
        np.linalg.eigh = orig


# --- Single qubit closed forms ----------------------------------------------------------
def _frozen(inst, s):
    A, B = model.schedule(inst, s)
    return dict(sched_s=np.array([0.0, 1.0]), sched_A=np.array([A, A]), sched_B=np.array([B, B]))


def test_single_qubit_no_bath_closed_form_propagator():
    inst = W.tfim_instance(1, 21, eta_g2=0.0, lamb_shift=False)
    for s in [0.1, 0.5, 0.9]:
        fr = lindblad.Frame(inst, s)
        A, B = model.schedule(inst, s)
        H = A * -model.SX + B * inst.hz[0] * model.SZ
        Om = math.hypot(A, B * inst.hz[0])
        t = 0.37
        U = math.cos(Om * t) * np.eye(2) - 1j * math.sin(Om * t) * H / Om
        assert np.max(np.abs(trajectories.Piece(fr, t).U_tau - U)) < 1e-14


def test_single_qubit_bath_closed_form_relaxation():
    inst = W.tfim_instance(1, 22, eta_g2=0.03)
    fr = lindblad.Frame(inst, 0.6)
    M = fr.M[0]
    D = fr.eig.evals[1] - fr.eig.evals[0]
    g = lambda w: bath.gamma(w, inst.eta_g2, inst.omega_c, inst.beta)  # noqa: E731
    down, up = g(D) * M[0, 1] ** 2, g(-D) * M[0, 1] ** 2
    deph = 0.5 * g(0.0) * (M[0, 0] - M[1, 1]) ** 2
    S = lambda w: bath.lamb_shift(w, inst.eta_g2, inst.omega_c, inst.beta, wmax=50.0)  # noqa: E731
    e0 = fr.eig.evals[0] + S(0.0) * (M[0, 0] ** 2) + S(-D) * M[1, 0] ** 2
    e1 = fr.eig.evals[1] + S(0.0) * (M[1, 1] ** 2) + S(D) * M[0, 1] ** 2
    rho = np.array([[0.3, 0.2 + 0.1j], [0.2 - 0.1j, 0.7]])
    t = 7.0
    out = fr.propagate(rho, t)
    p0_inf = down / (up + down)
    p0 = p0_inf + (0.3 - p0_inf) * math.exp(-(up + down) * t)
    coh = (0.2 + 0.1j) * np.exp((-1j * (e0 - e1) - 0.5 * (up + down) - deph) * t)
    assert abs(out[0, 0] - p0) < 1e-13
    assert abs(out[0, 1] - coh) < 1e-13
    assert abs(p0_inf / (1 - p0_inf) - math.exp(inst.beta * D)) < 1e-12 * math.exp(inst.beta * D)


def test_split_converges_second_order_without_bath():
    """g = 0: no jumps; the split propagation converges at O(dt^2) to an
    independent high-accuracy ODE solution of the Schroedinger equation."""
    inst = W.tfim_instance(2, 23, eta_g2=0.0, lamb_shift=False, t_f=2.0)
    HX, HZ = model.hamiltonian_terms(inst)

    def rhs(t, y):
        A, B = model.schedule(inst, t / inst.t_f)
        return -1j * ((A * HX + B * HZ) @ y)
    psi0 = model.eigen_at(inst, 0.0).V[:, 0].astype(complex)
    ref = integrate.solve_ivp(rhs, (0, inst.t_f), psi0, method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
    errs = []
    for K in (41, 81, 161):
        inst.n_grid = K
        p, jumps, fin = trajectories.sample(inst, [0])
        assert not jumps
        errs.append(1 - abs(np.vdot(ref, fin[0])))
    r1 = math.sqrt(errs[0] / errs[1])
    r2 = math.sqrt(errs[1] / errs[2])
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7


# --- Jump process ----------------------------------------------------------------------------
def test_eigenstate_has_no_drift():
    # App. E: a nondegenerate eigenstate only loses norm under H_eff.
    inst = W.tfim_instance(3, 24, eta_g2=0.05)
    fr = lindblad.Frame(inst, 0.5)
    pc = trajectories.Piece(fr, 0.8)
    for b in (0, 3):
        v = pc.U_tau @ fr.eig.V[:, b]
        c = fr.eig.V.T @ v
        others = np.delete(np.abs(c), b)
        assert np.max(others) < 1e-14
        assert abs(np.vdot(v, v).real - math.exp(2 * fr.K[b, b].imag * 0.8)) < 1e-14


def test_dephasing_jump_is_incomplete():
    # Sec. V.B: the omega = 0 operator reweights a superposition instead of projecting.
    inst = W.tfim_instance(2, 25, eta_g2=0.05)
    fr = lindblad.Frame(inst, 0.5)
    c = np.array([0.6, 0.8j, 0.0, 0.0])
    psi = fr.eig.V @ c
    # find u1 that lands on a dephasing unit (alpha, m={b}, a=b)
    for u1 in np.linspace(0.001, 0.999, 400):
        al, m, a, cls, new = trajectories.choose_jump(fr, psi, u1, 0.5)
        if cls == 0:
            break
    assert cls == 0
    expect = np.diag(fr.M[al]) * c
    expect /= np.linalg.norm(expect)
    got = fr.eig.V.T @ new
    assert np.max(np.abs(got - expect)) < 1e-14
    assert np.abs(got[0]) > 0.1 and np.abs(got[1]) > 0.1


@pytest.mark.parametrize("s", [0.0, 0.4])
def test_channel_frequencies_match_Pi(s):
    """App. B.1, Eq. Pi(t): channel i is chosen with probability <A_i^dag A_i>/lambda.
    The reference probabilities use dense operators built from eigenspace
    projectors in the computational basis (Eq. Lindblad2 written out)."""
    inst = W.tfim_instance(2, 26, eta_g2=0.05)
    fr = lindblad.Frame(inst, s)
    eig = fr.eig
    g = np.random.default_rng(6)
    psi = g.normal(size=4) + 1j * g.normal(size=4)
    psi /= np.linalg.norm(psi)
    P = [eig.V[:, m] @ eig.V[:, m].T for m in eig.manifolds]
    ref = {}
    for al in range(2):
        Z = model.op_on(al, model.SZ, 2)
        for ci, (w, pairs) in enumerate(fr.classes):
            gw = bath.gamma(w, inst.eta_g2, inst.omega_c, inst.beta)
            L = sum(P[ma] @ Z @ P[mb] for ma, mb in pairs)
            ref[(al, ci)] = gw * np.linalg.norm(L @ psi) ** 2
    tot = sum(ref.values())
    counts = {}
    n = 4000
    rng = np.random.default_rng(7)
    for _ in range(n):
        al, m, a, cls, _ = trajectories.choose_jump(fr, psi, rng.random(), rng.random())
        counts[(al, cls)] = counts.get((al, cls), 0) + 1
    assert set(counts) <= {k for k in ref if ref[k] > 0}
    big = [k for k in ref if ref[k] / tot * n >= 5]        # chi^2 bins, the rest pooled
    obs = np.array([counts.get(k, 0) for k in big] + [n - sum(counts.get(k, 0) for k in big)])
    pr = np.array([ref[k] / tot for k in big] + [1 - sum(ref[k] for k in big) / tot])
    keep = pr * n >= 1e-9
    obs, exp = obs[keep], (pr * n)[keep]
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    keys = obs
    assert stats.chi2.sf(chi2, len(keys) - 1) > 1e-3


def test_waiting_time_is_exponential():
    """App. C: from an eigenstate at frozen s the first jump time is exponential
    with rate -2 Im K_bb (the total rate out of level b, dephasing included)."""
    inst = W.tfim_instance(1, 27, eta_g2=0.08, t_f=40.0, n_grid=41, lamb_shift=False)
    f = _frozen(inst, 0.5)
    inst.sched_s, inst.sched_A, inst.sched_B = f["sched_s"], f["sched_A"], f["sched_B"]
    fr = lindblad.Frame(inst, 0.5)
    rate = -2 * fr.K[0, 0].imag
    p, jumps, _ = trajectories.sample(inst, range(600))
    first = {}
    for j in jumps:
        first.setdefault(j["traj"], j["t"])
    t = np.array(list(first.values()))
    # truncated exponential on [0, t_f]
    cdf = lambda x: (1 - np.exp(-rate * x)) / (1 - math.exp(-rate * inst.t_f))  # noqa: E731
    assert stats.kstest(t, cdf).pvalue > 1e-3
    assert abs(len(t) / 600 - (1 - math.exp(-rate * inst.t_f))) < 4 * math.sqrt(0.25 / 600)


def test_trajectory_average_matches_density_matrix():
    """App. B.2: the trajectory average recovers the AME (3 sigma, Bonferroni over
    five pre-declared grid points)."""
    inst = W.tfim_instance(2, 28, eta_g2=0.03, t_f=5.0, n_grid=101, seed=99)
    ref = ame.run(inst)["p_gs"]
    M = 1500
    p, jumps, _ = trajectories.sample(inst, range(M))
    assert len(jumps) > 200
    for k in (20, 40, 60, 80, 100):
        mean = p[:, k].mean()
        se = p[:, k].std(ddof=1) / math.sqrt(M)
        assert abs(mean - ref[k]) < 3.5 * se + 1e-12, (k, mean, ref[k], se)


# --- Bohr-frequency classes (Sec. II, Eq. Lindblad2) ----------------------------------------
# At s = 0 of the linear schedule H_S = -A sum sx with A = 2 pi: the manifolds are
# k = 0..n (k spins anti-aligned with the field), energy -A (n - 2k), multiplicity
# C(n, k), so the Bohr frequency of (m_a, m_b) is 2 A (k_b - k_a). The classes
# below are written out by hand from that arithmetic: (m_a, m_b) pairs, classes
# in increasing frequency, zero-frequency class first.
S0_CLASSES = {
    2: [(0, [(0, 0), (1, 1), (2, 2)]),
        (-2, [(2, 0)]),
        (-1, [(1, 0), (2, 1)]),
        (1, [(0, 1), (1, 2)]),
        (2, [(0, 2)])],
    3: [(0, [(0, 0), (1, 1), (2, 2), (3, 3)]),
        (-3, [(3, 0)]),
        (-2, [(2, 0), (3, 1)]),
        (-1, [(1, 0), (2, 1), (3, 2)]),
        (1, [(0, 1), (1, 2), (2, 3)]),
        (2, [(0, 2), (1, 3)]),
        (3, [(0, 3)])],
}


def _classes_as_sets(classes, unit):
    return [(round(w / unit), sorted(map(tuple, pairs))) for w, pairs in classes]


@pytest.mark.parametrize("n", [2, 3])
def test_bohr_classes_at_s0_written_out(n):
    inst = W.tfim_instance(n, 40 + n)
    eig = model.eigen_at(inst, 0.0)
    A = 2 * math.pi
    got = model.bohr_classes(eig)
    for w, _ in got:
        assert abs(w / (2 * A) - round(w / (2 * A))) < 1e-12
    assert _classes_as_sets(got, 2 * A) == [(w, sorted(p)) for w, p in S0_CLASSES[n]]


def test_bohr_classes_merge_distinct_pairs_of_equal_frequency():
    # s = 1 with hz = (1, 1/2), J = 0: levels -3/2, -1/2, 1/2, 3/2 (x 2 pi), all
    # nondegenerate and equally spaced, so distinct level pairs share each Bohr
    # frequency: omega = 2 pi has three pairs, 4 pi two, 6 pi one.
    inst = W.tfim_instance(2, 1)
    inst.hz = np.array([1.0, 0.5])
    inst.J = np.zeros((2, 2))
    eig = model.eigen_at(inst, 1.0)
    assert eig.nondegenerate
    got = _classes_as_sets(model.bohr_classes(eig), 2 * math.pi)
    assert got == [(0, [(0, 0), (1, 1), (2, 2), (3, 3)]),
                   (-3, [(3, 0)]),
                   (-2, [(2, 0), (3, 1)]),
                   (-1, [(1, 0), (2, 1), (3, 2)]),
                   (1, [(0, 1), (1, 2), (2, 3)]),
                   (2, [(0, 2), (1, 3)]),
                   (3, [(0, 3)])]


def _fourier_component(H, A, w, T=1e9):
    """(1/T) int_0^T e^{i w t} e^{iHt} A e^{-iHt} dt in closed form from the
    eigendecomposition of H (each matrix element oscillates at a difference of
    two eigenvalues): no tolerance-based grouping of frequencies is involved."""
    e, U = np.linalg.eigh(H)
    Ae = U.T @ A @ U
    d = w + e[:, None] - e[None, :]           # frequency of <a| ... |b> times e^{i w t}
    avg = np.where(np.abs(d) * T < 1e-3, 1.0 + 0j,
                   (np.exp(1j * np.clip(d * T, -1e300, 1e300)) - 1) / (1j * np.where(d == 0, 1, d) * T))
    return U @ (Ae * avg) @ U.T


@pytest.mark.parametrize("case", ["s0_n3", "equal_spacing", "generic"])
def test_class_operators_are_fourier_components(case):
    """Eq. Lindblad2: L_{alpha,omega} = sum over the class of P_a sz_alpha P_b is
    the omega-Fourier component of e^{iHt} sz_alpha e^{-iHt}. Checked against
    the time average computed independently, with sum_omega L = sz_alpha and
    [H, L] = -omega L. A class split in two, or two frequencies merged, fails."""
    if case == "s0_n3":
        inst, s = W.tfim_instance(3, 41), 0.0
    elif case == "equal_spacing":
        inst, s = W.tfim_instance(2, 1), 1.0
        inst.hz, inst.J = np.array([1.0, 0.5]), np.zeros((2, 2))
    else:
        inst, s = W.tfim_instance(3, 42), 0.4
    n = inst.n_qubits
    HX, HZ = model.hamiltonian_terms(inst)
    Aa, Bb = model.schedule(inst, s)
    H = Aa * HX + Bb * HZ
    eig = model.eigen_at(inst, s)
    P = [eig.V[:, m] @ eig.V[:, m].T for m in eig.manifolds]
    classes = model.bohr_classes(eig)
    ws = [w for w, _ in classes]
    assert all(abs(a - b) > 1e-6 for i, a in enumerate(ws) for b in ws[i + 1:])   # one class per frequency
    for al in range(n):
        Z = model.op_on(al, model.SZ, n)
        total = np.zeros_like(Z)
        for w, pairs in classes:
            L = sum(P[ma] @ Z @ P[mb] for ma, mb in pairs)
            total = total + L
            assert np.max(np.abs(H @ L - L @ H + w * L)) < 1e-10
            assert np.max(np.abs(_fourier_component(H, Z, w) - L)) < 1e-8
        assert np.max(np.abs(total - Z)) < 1e-12


def test_continuous_ame_converges_to_split_at_second_order():
    """The split-exact AME on the grid converges to the AME integrated without
    a grid (generator rebuilt at every integrator stage) at O(dt^2), bath on."""
    inst = W.tfim_instance(2, 28, eta_g2=0.03, t_f=5.0, n_grid=21, seed=99)
    cont = ame.run_continuous(inst)["p_gs"]
    errs = []
    for K in (21, 41, 81):
        inst.n_grid = K
        split = ame.run(inst)["p_gs"][:: (K - 1) // 20]
        errs.append(np.max(np.abs(split - cont)))
    assert errs[0] > 1e-4
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4


def test_grid_timing_jumps_at_the_end_of_the_refined_piece():
    """GRID timing (the norm condition of Sec. IV checked at time-step
    resolution): with the same random streams, the first jump of a trajectory
    comes at the end of the frozen piece that holds its refined jump time, with
    the same qubit (the state before it is the same)."""
    inst = W.tfim_instance(2, 28, eta_g2=0.03, t_f=5.0, n_grid=101, seed=99)
    M = 60
    _, jr, _ = trajectories.sample(inst, range(M))
    _, jg, _ = trajectories.sample(inst, range(M), timing="grid")
    tau = 0.5 * inst.t_f / (inst.n_grid - 1)
    fr = {}
    for j in jr:
        fr.setdefault(j["traj"], j)
    fg = {}
    for j in jg:
        fg.setdefault(j["traj"], j)
    assert set(fr) == set(fg) and len(fr) > 20
    for t, a in fr.items():
        b = fg[t]
        assert (a["grid"], a["half"]) == (b["grid"], b["half"])
        end = (math.floor(a["t"] / tau + 1e-9) + 1) * tau
        assert abs(b["t"] - end) < 1e-12
    for j in jg:   # every GRID jump sits on a piece boundary
        assert abs(j["t"] / tau - round(j["t"] / tau)) < 1e-9


# --- Fixed-step unravelling (App. B.1) ---------------------------------------------------------
def test_fixed_step_first_jump_is_geometric():
    """App. B.1: in each time step a jump happens with probability
    Delta p = dt lambda. From an eigenstate at frozen s (lambda constant until
    the first jump) the step of the first jump is geometric with parameter
    tau lambda, lambda = -2 Im K_bb."""
    inst = W.tfim_instance(1, 27, eta_g2=0.08, t_f=40.0, n_grid=41, lamb_shift=False)
    f = _frozen(inst, 0.5)
    inst.sched_s, inst.sched_A, inst.sched_B = f["sched_s"], f["sched_A"], f["sched_B"]
    fr = lindblad.Frame(inst, 0.5)
    tau = 0.5 * inst.t_f / (inst.n_grid - 1)
    pj = tau * (-2 * fr.K[0, 0].imag)
    M = 3000
    _, jumps, _ = trajectories.sample_fixed_step(inst, range(M))
    first = {}
    for j in jumps:
        if j["traj"] not in first:
            first[j["traj"]] = int(round(j["t"] / tau))    # piece index of the first jump
    npieces = 2 * (inst.n_grid - 1)
    counts = np.bincount(list(first.values()), minlength=npieces)[:npieces]
    # pool the pieces into 8 bins of equal width against the geometric law
    edges = np.linspace(0, npieces, 9).astype(int)
    obs = [counts[a:b].sum() for a, b in zip(edges[:-1], edges[1:])] + [M - len(first)]
    q = np.arange(npieces)
    pq = (1 - pj) ** q * pj
    exp = [M * pq[a:b].sum() for a, b in zip(edges[:-1], edges[1:])] + [M * (1 - pj) ** npieces]
    chi2 = float(np.sum((np.array(obs) - np.array(exp)) ** 2 / np.array(exp)))
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-3, (obs, exp)


def test_fixed_step_average_matches_density_matrix():
    """The fixed-step unravelling averages to the AME up to its O(dt) bias
    (App. B.1); with tau lambda ~ 1e-3 the bias is far below the statistical
    error at M = 1500 (3.5 sigma, sigma >= sqrt(p (1 - p) / M))."""
    inst = W.tfim_instance(2, 28, eta_g2=0.03, t_f=5.0, n_grid=201, seed=99)
    ref = ame.run(inst)["p_gs"]
    M = 1500
    p, jumps, _ = trajectories.sample_fixed_step(inst, range(M))
    assert len(jumps) > 500
    for k in (40, 80, 120, 160, 200):
        mean = p[:, k].mean()
        se = max(p[:, k].std(ddof=1) / math.sqrt(M), math.sqrt(ref[k] * (1 - ref[k]) / M))
        assert abs(mean - ref[k]) < 3.5 * se, (k, mean, ref[k], se)


# --- Truncated model (lowest levels only; a reading for the 16-qubit use) ------------------
def test_truncation_cut_follows_s0_multiplicities():
    """At s = 0 the levels of -A sum sx have multiplicities C(n, k): a cut is
    allowed only at the cumulative sums 1, 1 + n, 1 + n + C(n, 2), ..."""
    inst = W.tfim_instance(3, 5, n_grid=3)
    allowed = set(np.cumsum([math.comb(3, k) for k in range(4)]).tolist())  # {1, 4, 7, 8}
    for keep in range(1, 9):
        inst.n_levels = keep
        if keep in allowed:
            eig = model.eigen_at(inst, 0.0)
            assert eig.V.shape == (8, keep) and eig.truncated == (keep < 8)
        else:
            with pytest.raises(ValueError):
                model.eigen_at(inst, 0.0)


def test_truncated_first_frame_change_leaks_the_dropped_weight():
    """No bath: the first frame change of the truncated sampler moves out of the
    kept levels exactly the weight of the new frame's dropped levels in the
    initial ground state, computed here from the full eigensystems."""
    n, keep = 3, 4
    inst = W.tfim_instance(n, 7, eta_g2=0.0, t_f=4.0, n_grid=3, seed=1, n_levels=keep)
    _, jumps, _, leak = trajectories.sample(inst, [0, 1], return_leak=True)
    assert not jumps
    HX, HZ = model.hamiltonian_terms(inst)
    e0, V0 = np.linalg.eigh(2 * math.pi * HX)                       # s = 0
    e1, V1 = np.linalg.eigh(2 * math.pi * (0.5 * HX + 0.5 * HZ))    # s = 1/2
    want = float(np.sum((V1[:, keep:].T @ V0[:, 0]) ** 2))
    assert want > 1e-6
    np.testing.assert_allclose(leak[:, 1], want, rtol=1e-10)


def test_truncation_keeping_every_level_is_the_full_model():
    inst = W.tfim_instance(2, 28, eta_g2=0.03, t_f=3.0, n_grid=21, seed=9)
    full = ame.run(inst)
    inst.n_levels = 4
    same = ame.run(inst)
    np.testing.assert_array_equal(full["p_gs"], same["p_gs"])
    assert np.all(same["leak"] == 0.0)


def test_truncated_trajectory_average_matches_truncated_density_matrix():
    """The truncated sampler averages to the truncated AME (projected and
    renormalised at each frame change) within 3.5 sigma at four grid points;
    the per-trajectory renormalisation differs from the ensemble one only at
    second order in the leakage, which is ~1e-4 here."""
    inst = W.tfim_instance(3, 45, eta_g2=0.05, t_f=4.0, n_grid=41, seed=3, n_levels=4)
    ref = ame.run(inst)
    assert 1e-6 < ref["leak"].max() < 1e-2
    M = 600
    p, jumps, _, leak = trajectories.sample(inst, range(M), return_leak=True)
    assert len(jumps) > 50
    for k in (10, 20, 30, 40):
        mean = p[:, k].mean()
        se = max(p[:, k].std(ddof=1), 1e-3) / math.sqrt(M)
        assert abs(mean - ref["p_gs"][k]) < 3.5 * se, (k, mean, ref["p_gs"][k], se)
