"""Tensor-core (tcgen05, split-FP16) path against the FP64 oracle and the FP64
GPU path, through the C ABI.

The rotation runs as O_hi C_hi + O_hi C_lo + O_lo C_hi with FP32 accumulation
(22-bit mantissa), the state is FP32; the jump clock, crossing time and both
channel CDFs are FP64. With common random numbers every trajectory is expected
to keep the oracle's jump sequence; one whose draw sits within the FP32
state's rounding of a CDF boundary may diverge, so parity is asserted on the
identical ones (at least 97 %) and statistically on all.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import ame
from test_gpu_parity import compare_crn, run_lib, se_bound

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,M,grid,eta", [(7, 40, 101, 0.02), (8, 24, 41, 0.01)])
def test_tc_against_oracle(aqt_lib, n, M, grid, eta):
    """N = 128 and 256; ragged M (not a multiple of the 8-trajectory tile)."""
    inst = W.tfim_instance(n, 100 + n, eta_g2=eta, t_f=5.0, n_grid=grid, seed=21)
    res = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_F16SPLIT, M=M)
    assert res["status"] == aqt_lib.AQT_OK
    # jump times: FP64 root of the FP32 state's decay, clock from FP32 epilogue sums (measured <= 8e-8 ns)
    p, oj, _ = compare_crn(inst, res, list(range(M)), t_tol=1e-6, state_tol=1e-6, min_identical=0.97)
    assert len(oj) > 0
    assert np.max(np.abs(res["s1"] - p.sum(axis=0))) < 2e-4 * M


def test_tc_matches_fp64_gpu(aqt_lib):
    """Same instance, same streams: split-FP16 tensor-core run vs FP64 SIMT run."""
    inst = W.tfim_instance(7, 207, eta_g2=0.02, t_f=8.0, n_grid=301, seed=5)
    M = 300
    r64 = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_FP64, M=M)
    rtc = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_F16SPLIT, M=M)
    assert rtc["status"] == aqt_lib.AQT_OK
    j64 = {}
    for r in r64["jumps"]:
        j64.setdefault(int(r["traj"]), []).append((r["grid"], r["half"], r["alpha"], r["src"], r["dst"]))
    jtc = {}
    for r in rtc["jumps"]:
        jtc.setdefault(int(r["traj"]), []).append((r["grid"], r["half"], r["alpha"], r["src"], r["dst"]))
    same = [t for t in range(M) if j64.get(t, []) == jtc.get(t, [])]
    assert len(same) >= 0.97 * M
    ov = np.abs(np.einsum("mi,mi->m", r64["final"][same].conj(), rtc["final"][same]))
    assert np.max(np.abs(ov - 1.0)) < 1e-6
    t64 = {int(r["traj"]): [] for r in r64["jumps"]}
    for r in r64["jumps"]:
        t64[int(r["traj"])].append(r["t"])
    ttc = {}
    for r in rtc["jumps"]:
        ttc.setdefault(int(r["traj"]), []).append(r["t"])
    dts = [abs(a - b) for t in same for a, b in zip(t64.get(t, []), ttc.get(t, []))]
    assert max(dts) < 1e-5            # measured 1.9e-6 ns over 300 trajectories x 300 steps
    assert np.median(dts) < 1e-7      # measured 1.5e-8 ns
    assert np.max(np.abs(rtc["s1"] - r64["s1"])) < 1e-3 * M


def test_tc_against_ame(aqt_lib):
    inst = W.tfim_instance(7, 307, eta_g2=0.03, t_f=6.0, n_grid=151, seed=8)
    M = 1200
    res = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_F16SPLIT, M=M)
    ref = ame.run(inst)["p_gs"]
    for k in (50, 100, 150):
        assert abs(res["mean"][k] - ref[k]) < 3.5 * max(res["se"][k], se_bound(ref[k], M)), (k, res["mean"][k], ref[k])


def test_tc_rejects_small_n(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(6, 3, n_grid=5)
    c = A.aqt_create(0)
    A.aqt_set_ising(c, inst.n_qubits, inst.hz, inst.J)
    A.aqt_set_schedule(c, inst.sched_s, inst.sched_A, inst.sched_B)
    A.aqt_set_bath(c, inst.eta_g2, inst.omega_c, inst.beta, inst.lamb_shift)
    A.aqt_set_grid(c, inst.t_f, inst.n_grid)
    A.aqt_set_trajectories(c, 10, 1, A.AQT_PREC_F16SPLIT, 0, 16)
    with pytest.raises(A.AqtError) as e:
        A.aqt_workspace_size(c)
    assert e.value.status == A.AQT_EINVAL
    A.aqt_destroy(c)


def test_tc_general_jumps_at_degenerate_start(aqt_lib):
    """Jumps while the generator is frozen at s = 0, where H_S(0) has degenerate
    manifolds: the tensor-core kernel resolves them with the general FP64 jump
    routine. Against the FP64 GPU path (same streams) and the oracle."""
    A = aqt_lib
    inst = W.tfim_instance(7, 31, eta_g2=0.05, beta=0.15, t_f=2.0, n_grid=9, seed=5)
    M = 96
    r64 = run_lib(A, inst, A.AQT_PREC_FP64, M=M)
    rtc = run_lib(A, inst, A.AQT_PREC_F16SPLIT, M=M)
    assert rtc["status"] == A.AQT_OK and r64["status"] == A.AQT_OK
    at0 = rtc["jumps"][rtc["jumps"]["grid"] == 0]
    assert len(at0) >= 5
    j64, jtc = {}, {}
    for src, dst in ((r64, j64), (rtc, jtc)):
        for r in src["jumps"]:
            dst.setdefault(int(r["traj"]), []).append((r["grid"], r["half"], r["alpha"], r["src"], r["dst"]))
    same = [t for t in range(M) if j64.get(t, []) == jtc.get(t, [])]
    assert len(same) >= 0.9 * M
    ov = np.abs(np.einsum("mi,mi->m", r64["final"][same].conj(), rtc["final"][same]))
    assert np.max(np.abs(ov - 1.0)) < 2e-5
    compare_crn(inst, rtc, list(range(12)), t_tol=1e-6, state_tol=1e-6, min_identical=0.8)


def test_tc_wait_timeout_reports_and_recovers(aqt_lib):
    """A bounded wait made to expire (poll limit 0): the run ends with
    AQT_ETIMEOUT naming the wait, having issued no products; the same context
    then runs normally and reproduces a fresh context's result."""
    A = aqt_lib
    inst = W.tfim_instance(7, 207, eta_g2=0.02, t_f=8.0, n_grid=41, seed=5)
    S = A.Session(inst, precision=A.AQT_PREC_F16SPLIT, M=64)
    S.build()
    A.aqt_set_wait_limit(S.ctx, 0)
    A.aqt_run(S.ctx, S.stream())
    with pytest.raises(A.AqtError) as e:
        A.aqt_sync(S.ctx)
    assert e.value.status == A.AQT_ETIMEOUT and "B operand ready" in str(e.value)
    A.aqt_set_wait_limit(S.ctx, 1 << 22)
    assert S.run() == A.AQT_OK
    s1, s2 = A.aqt_get_observable_sums(S.ctx, inst.n_grid)
    fin = S.final_state(basis=0)
    S.close()
    T = A.Session(inst, precision=A.AQT_PREC_F16SPLIT, M=64)
    T.build()
    assert T.run() == A.AQT_OK
    t1, t2 = A.aqt_get_observable_sums(T.ctx, inst.n_grid)
    assert np.array_equal(s1, t1) and np.array_equal(s2, t2)
    assert np.array_equal(fin, T.final_state(basis=0))
    T.close()


def test_tc_grid_timing_matches_fp64(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(7, 207, eta_g2=0.02, t_f=8.0, n_grid=301, seed=5)
    M = 200
    r64 = run_lib(A, inst, A.AQT_PREC_FP64, M=M, timing=A.AQT_JUMP_GRID)
    rtc = run_lib(A, inst, A.AQT_PREC_F16SPLIT, M=M, timing=A.AQT_JUMP_GRID)
    assert rtc["status"] == A.AQT_OK
    tau = 0.5 * inst.t_f / (inst.n_grid - 1)
    assert np.all(np.abs(rtc["jumps"]["t"] / tau - np.round(rtc["jumps"]["t"] / tau)) < 1e-6)
    j64, jtc = {}, {}
    for src, dst in ((r64, j64), (rtc, jtc)):
        for r in src["jumps"]:
            dst.setdefault(int(r["traj"]), []).append((r["grid"], r["half"], r["alpha"], r["src"], r["dst"]))
    same = [t for t in range(M) if j64.get(t, []) == jtc.get(t, [])]
    assert len(same) >= 0.95 * M

