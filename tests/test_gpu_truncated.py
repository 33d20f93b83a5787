"""Truncated model (aqt_set_levels: only the lowest instantaneous levels are
kept) on the GPU against the oracle's truncated sampler, through the C ABI.

The library finds the kept eigenpairs with its FP64 Chebyshev-filtered block
solver (no dense eigensystem), the oracle with a dense one; with common
random numbers the jump sequences, final states (computational basis),
observable sums and per-step leakage sums must agree trajectory by
trajectory within the tolerances of each precision.
"""
import numpy as np
import pytest

import workloads as W
from oracle import trajectories
from test_gpu_parity import jumps_by_traj

pytestmark = pytest.mark.gpu


def _run(A, inst, precision, M):
    S = A.Session(inst, precision=precision, M=M)
    S.build()
    st = S.run()
    s1, _ = A.aqt_get_observable_sums(S.ctx, inst.n_grid)
    leak = A.aqt_get_leakage(S.ctx, inst.n_grid)
    jumps, dropped = S.jumps()
    final = S.final_state(basis=1)
    eig0 = S.final_state(basis=0)
    roterr = A.aqt_get_rotation_error(S.ctx)
    S.close()
    return dict(status=st, s1=s1, leak=leak, jumps=jumps, dropped=dropped, final=final, eig0=eig0, roterr=roterr)


def _compare(inst, res, M, t_tol, state_tol, min_identical):
    p, oj, ofin, oleak = trajectories.sample(inst, list(range(M)), return_leak=True)
    gj, ojt = jumps_by_traj(res["jumps"]), jumps_by_traj(oj)
    identical = 0
    for t in range(M):
        a, b = gj.get(t, []), ojt.get(t, [])
        same = len(a) == len(b) and all(
            (x["grid"], x["half"], x["alpha"], x["src"], x["dst"]) ==
            (y["grid"], y["half"], y["alpha"], y["src"], y["dst"]) and abs(x["t"] - y["t"]) <= t_tol
            for x, y in zip(a, b))
        if same:
            identical += 1
            ov = abs(np.vdot(res["final"][t], ofin[t]))
            assert abs(ov - 1.0) <= state_tol, (t, ov)
    assert identical >= min_identical * M, (identical, M)
    return p, oj, oleak


@pytest.mark.parametrize("n,levels,prec,M,grid,eta", [
    (6, 22, "FP64", 40, 41, 0.03),   # 1 + 6 + 15 levels: the s = 0 manifolds up to two flipped spins
    (7, 29, "FP32", 40, 41, 0.03),   # 1 + 7 + 21
])
def test_truncated_against_oracle(aqt_lib, n, levels, prec, M, grid, eta):
    A = aqt_lib
    inst = W.tfim_instance(n, 300 + n, eta_g2=eta, t_f=4.0, n_grid=grid, seed=7, n_levels=levels)
    res = _run(A, inst, getattr(A, "AQT_PREC_" + prec), M)
    assert res["status"] == A.AQT_OK and res["dropped"] == 0
    assert res["eig0"].shape == (M, levels) and res["final"].shape == (M, 1 << n)
    fp64 = prec == "FP64"
    p, oj, oleak = _compare(inst, res, M, t_tol=1e-10 if fp64 else 1e-7, state_tol=1e-10 if fp64 else 1e-6,
                            min_identical=1.0 if fp64 else 0.97)
    assert len(oj) > 5
    np.testing.assert_allclose(res["s1"], p.sum(axis=0), rtol=0, atol=(2e-10 if fp64 else 2e-4) * M)
    # leakage of each frame change, summed over trajectories (the oracle's
    # projections against the kernel's norm loss of the truncated rotation)
    ol = oleak.sum(axis=0)
    assert ol[1:].max() > 1e-6
    np.testing.assert_allclose(res["leak"], ol, rtol=0, atol=(1e-12 if fp64 else 2e-6) * M)
    assert res["roterr"] >= oleak.max() * 0.99


def test_truncated_tensor_cores_against_oracle(aqt_lib):
    """256 of the 512 levels of 9 qubits (1 + 9 + 36 + 84 + 126: the s = 0
    manifolds up to four flipped spins) on the tensor-core path."""
    A = aqt_lib
    inst = W.tfim_instance(9, 309, eta_g2=0.03, t_f=2.0, n_grid=7, seed=5, n_levels=256)
    M = 16
    res = _run(A, inst, A.AQT_PREC_F16SPLIT, M)
    assert res["status"] == A.AQT_OK
    p, oj, oleak = _compare(inst, res, M, t_tol=1e-6, state_tol=1e-5, min_identical=0.9)
    np.testing.assert_allclose(res["leak"], oleak.sum(axis=0), rtol=0, atol=1e-5 * M)


def test_twelve_qubits_truncated_properties(aqt_lib):
    """4096-dimensional space, 79 levels kept (no dense eigensystem anywhere):
    populations in [0, 1], small positive leakage, repeatable."""
    A = aqt_lib
    inst = W.tfim_instance(12, 312, eta_g2=0.01, t_f=4.0, n_grid=21, seed=3, n_levels=79)
    r1 = _run(A, inst, A.AQT_PREC_FP32, 64)
    r2 = _run(A, inst, A.AQT_PREC_FP32, 64)
    assert r1["status"] == A.AQT_OK
    mean = r1["s1"] / 64
    assert np.all(mean >= -1e-6) and np.all(mean <= 1 + 1e-6) and mean[0] == pytest.approx(1.0)
    assert np.all(r1["leak"][1:] >= -1e-4) and r1["leak"][1:].max() < 64 * 0.05
    assert np.array_equal(r1["s1"], r2["s1"]) and np.array_equal(r1["final"], r2["final"])
    nrm = np.linalg.norm(r1["final"], axis=1)
    np.testing.assert_allclose(nrm, 1.0, atol=1e-5)
