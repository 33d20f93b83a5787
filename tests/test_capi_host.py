"""Host-side checks of the C ABI (no GPU): symbols, argument validation, and
the FP64 tables built by the library against the oracle."""
import math
import re

import numpy as np
import pytest

import workloads as W
from oracle import lindblad


def _declared_symbols():
    hdr = open(__file__.replace("tests/test_capi_host.py", "include/aqt.h")).read()
    return sorted(set(re.findall(r"\b(aqt_[a-z_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol(aqt_lib):
    lib = aqt_lib.lib()
    syms = _declared_symbols()
    assert len(syms) >= 21
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(aqt_lib.EXPORTS)


def _host_ctx(A, inst, M=10, precision=0):
    c = A.aqt_create(-1)
    A.aqt_set_ising(c, inst.n_qubits, inst.hz, inst.J)
    A.aqt_set_schedule(c, inst.sched_s, inst.sched_A, inst.sched_B)
    A.aqt_set_bath(c, inst.eta_g2, inst.omega_c, inst.beta, inst.lamb_shift)
    A.aqt_set_grid(c, inst.t_f, inst.n_grid)
    A.aqt_set_trajectories(c, M, 1, precision, 0, 16)
    return c


def test_argument_validation(aqt_lib):
    A = aqt_lib
    c = A.aqt_create(-1)
    with pytest.raises(A.AqtError) as e:
        A.aqt_set_ising(c, 0, [1.0], [0.0])
    assert e.value.status == A.AQT_EINVAL
    with pytest.raises(A.AqtError):
        A.aqt_set_ising(c, 17, np.zeros(17), np.zeros(289))
    with pytest.raises(A.AqtError):
        A.aqt_set_levels(c, -1)
    with pytest.raises(A.AqtError):
        A.aqt_set_schedule(c, [0.0, 0.5], [1, 1], [0, 1])          # does not reach 1
    with pytest.raises(A.AqtError):
        A.aqt_set_schedule(c, [0.0, 0.6, 0.5, 1.0], [1] * 4, [0] * 4)
    with pytest.raises(A.AqtError):
        A.aqt_set_bath(c, 1e-3, 0.0, 1.0, 1)
    with pytest.raises(A.AqtError):
        A.aqt_set_grid(c, 10.0, 1)
    with pytest.raises(A.AqtError):
        A.aqt_set_trajectories(c, 0, 1, 0, 0, 10)
    with pytest.raises(A.AqtError):
        A.aqt_set_trajectories(c, 10, 1, 7, 0, 10)
    with pytest.raises(A.AqtError):
        A.aqt_workspace_size(c)                                       # inputs incomplete
    with pytest.raises(A.AqtError):
        A.aqt_set_ising(c, 2, [np.nan, 0.0], np.zeros(4))
    A.aqt_destroy(c)
    with pytest.raises(A.AqtError):
        A.aqt_create(-2)


def test_host_context_cannot_run(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(2, 3, n_grid=5)
    c = _host_ctx(A, inst)
    assert A.aqt_workspace_size(c) > 0
    A.aqt_build_tables(c, 0)
    with pytest.raises(A.AqtError) as e:
        A.aqt_run(c, 0)
    assert e.value.status == A.AQT_ENODEV
    A.aqt_destroy(c)


@pytest.mark.parametrize("n,seed,s_idx", [(3, 7, [0, 4, 10]), (4, 1710_03431, [0, 1, 7, 10])])
def test_tables_match_oracle(aqt_lib, n, seed, s_idx):
    A = aqt_lib
    inst = W.tfim_instance(n, seed, n_grid=11)
    N = 1 << n
    c = _host_ctx(A, inst)
    A.aqt_build_tables(c, 0)
    for g in s_idx:
        fr = lindblad.Frame(inst, g / 10)
        ev = A.aqt_debug_table(c, 0, g, (N,))
        np.testing.assert_allclose(ev, fr.eig.evals, atol=1e-12)
        kd = A.aqt_debug_table(c, 1, g, (N, 2))
        Kd = kd[:, 0] + 1j * kd[:, 1]
        np.testing.assert_allclose(Kd.imag, np.diag(fr.K).imag, atol=1e-13)
        np.testing.assert_allclose(Kd.real, np.diag(fr.K).real, atol=1e-8)   # Lamb-shift tables
        V = A.aqt_debug_table(c, 5, g, (N, N))
        assert np.max(np.abs(V.T @ V - np.eye(N))) < 1e-13
        H = V @ np.diag(ev) @ V.T
        Ho = fr.eig.V @ np.diag(fr.eig.evals) @ fr.eig.V.T
        assert np.max(np.abs(H - Ho)) < 1e-12
        if fr.eig.nondegenerate:
            Rl = A.aqt_debug_table(c, 3, g, (n, N, N))
            assert np.max(np.abs(np.abs(Rl) - np.abs(fr.R))) < 1e-12
            G = A.aqt_debug_table(c, 2, g, (n, N))
            Go = np.sum(fr.gam[None] * fr.M ** 2, axis=1)
            np.testing.assert_allclose(G, Go, rtol=1e-11, atol=1e-16)
        if g < 10:
            O = A.aqt_debug_table(c, 4, g, (N, N))
            V1 = A.aqt_debug_table(c, 5, g + 1, (N, N))
            assert np.max(np.abs(O - V1.T @ V)) < 1e-13
    A.aqt_destroy(c)


@pytest.mark.parametrize("n,levels,seed,s_idx", [(6, 22, 17, [0, 1, 6, 10]), (8, 37, 23, [0, 3, 10])])
def test_truncated_tables_match_oracle(aqt_lib, n, levels, seed, s_idx):
    """Tables of the truncated model (lowest levels only, eigenpairs from the
    library's matrix-free FP64 block solver) against the oracle's dense
    eigensystem restricted to the same levels."""
    A = aqt_lib
    inst = W.tfim_instance(n, seed, n_grid=11, n_levels=levels)
    N, D = levels, 1 << n
    c = _host_ctx(A, inst)
    A.aqt_set_levels(c, levels)
    A.aqt_build_tables(c, 0)
    for g in s_idx:
        fr = lindblad.Frame(inst, g / 10)
        ev = A.aqt_debug_table(c, 0, g, (N,))
        np.testing.assert_allclose(ev, fr.eig.evals, atol=1e-10)
        kd = A.aqt_debug_table(c, 1, g, (N, 2))
        Kd = kd[:, 0] + 1j * kd[:, 1]
        np.testing.assert_allclose(Kd.imag, np.diag(fr.K).imag, atol=1e-12)
        np.testing.assert_allclose(Kd.real, np.diag(fr.K).real, atol=1e-8)   # Lamb-shift tables
        V = A.aqt_debug_table(c, 5, g, (D, N))
        assert np.max(np.abs(V.T @ V - np.eye(N))) < 1e-12
        # the kept span and its spectral projector agree, whatever the basis inside
        # degenerate manifolds
        P, Po = V @ np.diag(ev) @ V.T, fr.eig.V @ np.diag(fr.eig.evals) @ fr.eig.V.T
        assert np.max(np.abs(P - Po)) < 1e-10
        nxt = A.aqt_debug_table(c, 9, g, (2,))[0]
        assert nxt > ev[-1] + 1e-6
        if fr.eig.nondegenerate:
            G = A.aqt_debug_table(c, 2, g, (n, N))
            Go = np.sum(fr.gam[None] * fr.M ** 2, axis=1)
            np.testing.assert_allclose(G, Go, rtol=1e-9, atol=1e-14)
        if g < 10:
            O = A.aqt_debug_table(c, 4, g, (N, N))
            V1 = A.aqt_debug_table(c, 5, g + 1, (D, N))
            assert np.max(np.abs(O - V1.T @ V)) < 1e-12
            sv = np.linalg.svd(O, compute_uv=False)
            assert sv.max() <= 1 + 1e-12 and sv.min() < 1  # a contraction that leaks
    A.aqt_destroy(c)


def test_truncation_splitting_a_manifold_rejected(aqt_lib):
    """At s = 0 the 6-qubit levels have multiplicities 1, 6, 15, ...: keeping
    20 levels would cut the 15-fold manifold."""
    A = aqt_lib
    inst = W.tfim_instance(6, 17, n_grid=5)
    c = _host_ctx(A, inst)
    A.aqt_set_levels(c, 20)
    with pytest.raises(A.AqtError) as e:
        A.aqt_build_tables(c, 0)
    assert e.value.status == A.AQT_EDEGEN and "splits" in str(e.value)
    A.aqt_destroy(c)


def test_eleven_qubits_need_truncation(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(11, 5, n_grid=3)
    c = _host_ctx(A, inst)
    with pytest.raises(A.AqtError) as e:
        A.aqt_build_tables(c, 0)
    assert e.value.status == A.AQT_EINVAL and "aqt_set_levels" in str(e.value)
    A.aqt_destroy(c)


def test_degenerate_ground_state_rejected(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(2, 3, n_grid=5)
    inst.sched_A = np.array([0.0, 0.0])       # H(0) = 0: fully degenerate start
    c = _host_ctx(A, inst)
    with pytest.raises(A.AqtError) as e:
        A.aqt_build_tables(c, 0)
    assert e.value.status == A.AQT_EDEGEN


@pytest.mark.parametrize("n,seed,grid,idx", [(3, 7, 11, [0, 1, 5, 10]), (4, 1710_03431, 201, [0, 1, 2, 50, 200])])
def test_grid_metadata_matches_oracle(aqt_lib, n, seed, grid, idx):
    """Manifold and Bohr-class bookkeeping that selects the jump operator's
    form: degenerate manifolds, ground-manifold size, and whether every class
    of nonzero frequency is one manifold pair (Eq. Lindblad2)."""
    from oracle import model
    A = aqt_lib
    inst = W.tfim_instance(n, seed, n_grid=grid)
    c = _host_ctx(A, inst)
    A.aqt_build_tables(c, 0)
    terms = model.hamiltonian_terms(inst)
    for g in idx:
        eig = model.eigen_at(inst, g / (grid - 1), terms)
        meta = A.aqt_debug_table(c, 7, g, (4,))
        classes = model.bohr_classes(eig)
        simple = all(len(pairs) == 1 for _, pairs in classes[1:])
        assert bool(meta[0]) == (not eig.nondegenerate), g
        assert int(meta[1]) == int(np.sum(eig.level_manifold == 0)), g
        assert bool(meta[2]) == simple, g
        assert meta[3] == pytest.approx(eig.tol, rel=1e-15), g
    A.aqt_destroy(c)


def test_device_run_sizes(aqt_lib):
    """SIMT runs take up to 512 levels (n = 9); the tensor-core path only
    N = 128 or 256."""
    A = aqt_lib
    inst = W.tfim_instance(9, 3, n_grid=3)
    c = _host_ctx(A, inst, precision=A.AQT_PREC_FP32)
    assert A.aqt_workspace_size(c) > 2 * 512 * 512 * 4  # eigenvectors and rotations of 3 grid points
    A.aqt_destroy(c)
    c = _host_ctx(A, inst, precision=A.AQT_PREC_F16SPLIT)
    with pytest.raises(A.AqtError) as e:
        A.aqt_workspace_size(c)
    assert e.value.status == A.AQT_EINVAL
    A.aqt_destroy(c)


def test_batch_needs_device_tables(aqt_lib):
    """A batch takes contexts whose tables are on a device; a host-only
    context (or none) is refused."""
    A = aqt_lib
    inst = W.tfim_instance(3, 5, n_grid=5)
    c = _host_ctx(A, inst)
    A.aqt_build_tables(c)
    for members in ([c], []):
        with pytest.raises(A.AqtError) as e:
            A.aqt_batch_create(members)
        assert e.value.status == A.AQT_EINVAL
    A.aqt_destroy(c)


def test_binding_fails_loudly_without_library(tmp_path):
    """No fallback: without the compiled library every entry point raises."""
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1710_03431_gb300 import aqt\n"
        "aqt.LIB_PATH = %r\n"
        "aqt._lib = None\n"
        "try:\n"
        "    aqt.aqt_create(0)\n"
        "except ImportError as e:\n"
        "    print('raised', e)\n"
    ) % (__file__.rsplit("/tests/", 1)[0], str(tmp_path / "libaqt.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "raised" in r.stdout and "missing" in r.stdout


def test_dt_condition_terms_and_warning(aqt_lib):
    """Eq. newcond (Sec. IV): the library's three terms against the oracle's
    generator, and AQT_WDT on a grid that is too coarse."""
    A = aqt_lib
    inst = W.tfim_instance(3, 7, t_f=10.0, n_grid=41)
    c = _host_ctx(A, inst)
    assert A.aqt_build_tables(c, 0) == A.AQT_OK
    b, at = A.aqt_get_dt_bounds(c)
    s = np.arange(inst.n_grid) / (inst.n_grid - 1)
    dt = inst.t_f / (inst.n_grid - 1)
    frames = [lindblad.Frame(inst, float(x)) for x in s]
    heff = [f.eig.V @ f.K @ f.eig.V.T for f in frames]
    hn = np.array([np.linalg.norm(h, 2) for h in heff])
    # 1/|H_eff| is exact: the operator norm of the oracle's H_eff
    assert b[1] == pytest.approx(1.0 / hn.max(), rel=1e-9)
    assert at[1] == int(np.argmax(hn))
    # 2|H_eff|/|dH_eff/dt| uses an upper estimate of the derivative: never above the
    # value with the exact finite-difference derivative, and not far below it
    hdot = np.array([np.linalg.norm(heff[g + 1] - heff[g], 2) / dt for g in range(inst.n_grid - 1)])
    fd = np.min(2 * hn[:-1] / hdot)
    assert b[0] <= fd * (1 + 1e-6) and b[0] > 0.2 * fd
    # lambda term per eigenstate: lambda_b = -2 Im K_bb
    lam = np.array([-2 * np.diag(f.K).imag for f in frames])
    ref = np.inf
    for g in range(inst.n_grid - 1):
        ld = (lam[g + 1] - lam[g]) / dt
        ok = lam[g] * inst.t_f > 1e-6
        ref = min(ref, np.min(np.abs(lam[g][ok] / (lam[g][ok] ** 2 - ld[ok]))))
    assert b[2] <= ref * (1 + 1e-6)
    A.aqt_destroy(c)
    coarse = W.tfim_instance(3, 7, t_f=10.0, n_grid=3)
    c = _host_ctx(A, coarse)
    assert A.aqt_build_tables(c, 0) == A.AQT_WDT
    assert "newcond" in A.aqt_last_error(c)
    A.aqt_destroy(c)


def test_gradient_entry_points_on_a_host_context(aqt_lib):
    """The parameter count needs the inputs only; the device calls of a
    gradient run refuse a host-only context."""
    A = aqt_lib
    inst = W.tfim_instance(3, 5, t_f=2.0, n_grid=20, M=8, seed=3)
    c = _host_ctx(A, inst, M=8)
    try:
        k = len(inst.sched_s)
        assert A.aqt_grad_n_params(c) == 2 * k + 3 + 3
        with pytest.raises(A.AqtError) as e:
            A.aqt_grad_workspace_size(c, 64, 1024)
        assert e.value.status == A.AQT_ENODEV
        with pytest.raises(A.AqtError) as e:
            A.aqt_grad_forward(c, 0)
        assert e.value.status == A.AQT_ENODEV
    finally:
        A.aqt_destroy(c)
    c = A.aqt_create(-1)
    try:
        with pytest.raises(A.AqtError) as e:
            A.aqt_grad_n_params(c)
        assert e.value.status == A.AQT_EINVAL
    finally:
        A.aqt_destroy(c)

