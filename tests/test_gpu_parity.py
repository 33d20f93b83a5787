"""CUDA path against the FP64 oracle, through the C ABI.

With the same Philox streams (common random numbers) the FP64 GPU path must
reproduce the oracle trajectory by trajectory: the same jumps (time, qubit,
source, target), the same final states and the same per-grid observable
sums. The FP32 path must match within FP32 tolerances, and both must agree
with the density-matrix AME within 3 standard errors.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import ame, trajectories

pytestmark = pytest.mark.gpu


def run_lib(A, inst, precision, M=None, jcap=None, timing=0):
    S = A.Session(inst, precision=precision, M=M, jump_capacity=jcap, timing=timing)
    S.build()
    status = S.run()
    mean, se = S.observables()
    s1, s2 = A.aqt_get_observable_sums(S.ctx, inst.n_grid)
    jumps, dropped = S.jumps()
    final = S.final_state(basis=1)
    roterr = A.aqt_get_rotation_error(S.ctx)
    S.close()
    return dict(status=status, mean=mean, se=se, s1=s1, s2=s2, jumps=jumps, dropped=dropped, final=final,
                roterr=roterr)


def se_bound(ref, M):
    """Upper bound on the standard error of a mean of M values in [0, 1] whose
    mean is ref: var <= ref (1 - ref). The sample error underestimates the true
    one when excitations are rare events (none may have happened yet)."""
    return math.sqrt(max(ref * (1.0 - ref), 0.0) / M)


def jumps_by_traj(recs):
    out = {}
    for r in recs:
        out.setdefault(int(r["traj"]), []).append(r)
    return out


def compare_crn(inst, res, traj_ids, t_tol, state_tol, min_identical=1.0, timing="refined"):
    """Oracle on traj_ids with the same streams; returns the oracle output."""
    p, ojumps, ofin = trajectories.sample(inst, traj_ids, timing=timing)
    gj = jumps_by_traj(res["jumps"])
    oj = jumps_by_traj(ojumps)
    identical = 0
    for i, t in enumerate(traj_ids):
        a, b = gj.get(t, []), oj.get(t, [])
        same = len(a) == len(b) and all(
            (x["grid"], x["half"], x["alpha"], x["src"], x["dst"]) ==
            (y["grid"], y["half"], y["alpha"], y["src"], y["dst"]) and abs(x["t"] - y["t"]) <= t_tol
            and abs(x["omega"] - y["omega"]) <= 1e-8 for x, y in zip(a, b))
        if same:
            identical += 1
            ov = abs(np.vdot(res["final"][t], ofin[i]))
            assert abs(ov - 1.0) <= state_tol, (t, ov)
    assert identical >= min_identical * len(traj_ids), (identical, len(traj_ids))
    return p, ojumps, ofin


def test_two_qubit_fp64_every_trajectory(aqt_lib):
    """Ragged M (not a multiple of the CTA tile), strong bath, many jumps."""
    inst = W.tfim_instance(2, 28, eta_g2=0.03, t_f=5.0, n_grid=101, seed=99)
    M = 37
    res = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_FP64, M=M)
    assert res["status"] == aqt_lib.AQT_OK and res["dropped"] == 0
    p, oj, _ = compare_crn(inst, res, list(range(M)), t_tol=1e-10, state_tol=1e-10)
    assert len(oj) > 10 and len(res["jumps"]) == len(oj)
    np.testing.assert_allclose(res["s1"], p.sum(axis=0), rtol=0, atol=1e-9)
    np.testing.assert_allclose(res["s2"], (p ** 2).sum(axis=0), rtol=0, atol=1e-9)


def test_degenerate_start_hot_bath_fp64(aqt_lib):
    """Jumps while the generator is frozen at s = 0, where H_S(0) has degenerate
    manifolds and Bohr classes with many level pairs (Eq. Lindblad2)."""
    inst = W.tfim_instance(2, 31, eta_g2=0.4, beta=0.15, t_f=2.0, n_grid=5, seed=5)
    M = 200
    res = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_FP64, M=M)
    assert res["status"] == aqt_lib.AQT_OK
    recs = res["jumps"]
    at0 = recs[recs["grid"] == 0]
    assert len(at0) > 50
    # a second jump from a degenerate manifold at s = 0
    assert np.any((at0["src"] == 1) | (at0["src"] == 2))
    p, oj, _ = compare_crn(inst, res, list(range(M)), t_tol=1e-10, state_tol=1e-9)
    np.testing.assert_allclose(res["s1"], p.sum(axis=0), atol=1e-8)


def test_three_qubit_fp64_and_ame(aqt_lib):
    inst = W.tfim_instance(3, 44, eta_g2=0.02, t_f=6.0, n_grid=201, seed=3)
    M = 300
    res = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_FP64, M=M)
    p, oj, _ = compare_crn(inst, res, list(range(M)), t_tol=1e-10, state_tol=1e-9)
    np.testing.assert_allclose(res["s1"], p.sum(axis=0), atol=1e-8)
    ref = ame.run(inst)["p_gs"]
    for k in (50, 100, 150, 200):
        assert abs(res["mean"][k] - ref[k]) < 3.5 * max(res["se"][k], se_bound(ref[k], M)) + 1e-9


def test_cfg_small_fp64_full(aqt_lib):
    """4 qubits, N = 16, 1000-point grid, t_f = 10 ns, M = 1000, complex128:
    every trajectory against the oracle, and the mean against the AME."""
    inst = W.cfg_small()
    res = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_FP64)
    assert res["status"] == aqt_lib.AQT_OK
    p, oj, _ = compare_crn(inst, res, list(range(inst.M)), t_tol=1e-9, state_tol=1e-9)
    assert len(res["jumps"]) == len(oj)
    np.testing.assert_allclose(res["s1"], p.sum(axis=0), atol=1e-8)
    ref = ame.run(inst)["p_gs"]
    pts = [250, 500, 750, 999]
    for k in pts:
        tol = 3.5 * max(res["se"][k], se_bound(ref[k], inst.M))
        assert abs(res["mean"][k] - ref[k]) < tol, (k, res["mean"][k], ref[k], tol)


def test_fp32_against_oracle(aqt_lib):
    inst = W.tfim_instance(3, 45, eta_g2=0.02, t_f=6.0, n_grid=201, seed=4)
    M = 300
    res = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_FP32, M=M)
    assert res["status"] == aqt_lib.AQT_OK
    p, oj, _ = compare_crn(inst, res, list(range(M)), t_tol=1e-7, state_tol=1e-6, min_identical=0.97)
    # observable sums: FP32 state, FP64 accumulation
    assert np.max(np.abs(res["s1"] - p.sum(axis=0))) < 1e-3 * M
    ref = ame.run(inst)["p_gs"]
    for k in (100, 200):
        assert abs(res["mean"][k] - ref[k]) < 3.5 * max(res["se"][k], se_bound(ref[k], M)) + 1e-6


def test_repeatable_and_overflow(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(2, 28, eta_g2=0.03, t_f=5.0, n_grid=51, seed=7)
    r1 = run_lib(A, inst, A.AQT_PREC_FP64, M=64)
    r2 = run_lib(A, inst, A.AQT_PREC_FP64, M=64)
    assert np.array_equal(r1["s1"], r2["s1"]) and np.array_equal(r1["final"], r2["final"])
    total = len(r1["jumps"])
    assert total > 0
    r3 = run_lib(A, inst, A.AQT_PREC_FP64, M=64, jcap=0)
    assert r3["status"] == A.AQT_EOVERFLOW and r3["dropped"] == total
    assert np.array_equal(r3["s1"], r1["s1"])


def test_minimal_sizes(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(1, 2, n_grid=2, t_f=0.5, seed=1)
    res = run_lib(A, inst, A.AQT_PREC_FP64, M=1)
    p, oj, _ = compare_crn(inst, res, [0], t_tol=1e-12, state_tol=1e-12)
    np.testing.assert_allclose(res["s1"], p.sum(axis=0), atol=1e-12)


def test_grid_timing_fp64_every_trajectory(aqt_lib):
    """GRID jump timing (jump at the end of the frozen half-step in which the
    norm fell to the threshold) against the oracle's GRID sampler."""
    inst = W.tfim_instance(2, 28, eta_g2=0.03, t_f=5.0, n_grid=101, seed=99)
    M = 37
    res = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_FP64, M=M, timing=aqt_lib.AQT_JUMP_GRID)
    assert res["status"] == aqt_lib.AQT_OK
    p, oj, _ = compare_crn(inst, res, list(range(M)), t_tol=1e-12, state_tol=1e-10, timing="grid")
    assert len(oj) > 10 and len(res["jumps"]) == len(oj)
    np.testing.assert_allclose(res["s1"], p.sum(axis=0), rtol=0, atol=1e-9)


def test_rotation_norm_error_fp64_fp32(aqt_lib):
    """P12 on the kernels' own arithmetic: the largest relative change of the
    squared norm over one frame rotation (1e-5 budget for FP32)."""
    inst = W.tfim_instance(6, 46, eta_g2=0.02, t_f=6.0, n_grid=201, seed=4)
    r64 = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_FP64, M=64)
    r32 = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_FP32, M=64)
    assert 0.0 < r64["roterr"] < 1e-12
    assert 0.0 < r32["roterr"] < 1e-5



def _compare_fixed_step(A, inst, res, M, t_tol, state_tol, min_identical):
    p, oj, ofin = trajectories.sample_fixed_step(inst, list(range(M)))
    gj, ojj = jumps_by_traj(res["jumps"]), jumps_by_traj(oj)
    identical = 0
    for t in range(M):
        a, b = gj.get(t, []), ojj.get(t, [])
        if len(a) == len(b) and all((x["grid"], x["half"], x["alpha"], x["src"], x["dst"]) ==
                                    (y["grid"], y["half"], y["alpha"], y["src"], y["dst"]) and
                                    abs(x["t"] - y["t"]) <= t_tol for x, y in zip(a, b)):
            identical += 1
            assert abs(abs(np.vdot(res["final"][t], ofin[t])) - 1.0) <= state_tol, t
    assert identical >= min_identical * M, (identical, M)
    return p, oj


def test_fixed_step_sampler_fp64_every_trajectory(aqt_lib):
    """The fixed-step unravelling of App. B.1 (a jump test with probability
    tau lambda per half-step) against the oracle's, same random streams."""
    A = aqt_lib
    inst = W.tfim_instance(2, 28, eta_g2=0.03, t_f=5.0, n_grid=101, seed=99)
    M = 64
    res = run_lib(A, inst, A.AQT_PREC_FP64, M=M, timing=A.AQT_JUMP_FIXED_STEP)
    assert res["status"] == A.AQT_OK
    p, oj = _compare_fixed_step(A, inst, res, M, t_tol=1e-12, state_tol=1e-10, min_identical=1.0)
    assert len(oj) > 10 and len(res["jumps"]) == len(oj)
    np.testing.assert_allclose(res["s1"], p.sum(axis=0), rtol=0, atol=1e-9)


def test_fixed_step_sampler_fp32_and_ame(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(3, 45, eta_g2=0.02, t_f=6.0, n_grid=201, seed=4)
    M = 300
    res = run_lib(A, inst, A.AQT_PREC_FP32, M=M, timing=A.AQT_JUMP_FIXED_STEP)
    assert res["status"] == A.AQT_OK
    _compare_fixed_step(A, inst, res, M, t_tol=1e-12, state_tol=1e-6, min_identical=0.97)
    ref = ame.run(inst)["p_gs"]
    for k in (100, 200):
        assert abs(res["mean"][k] - ref[k]) < 3.5 * max(res["se"][k], se_bound(ref[k], M)) + 1e-6


def test_fixed_step_sampler_not_on_tensor_cores(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(7, 3, n_grid=5)
    with pytest.raises(A.AqtError) as e:
        A.Session(inst, precision=A.AQT_PREC_F16SPLIT, M=16, timing=A.AQT_JUMP_FIXED_STEP).build()
    assert e.value.status == A.AQT_EINVAL
