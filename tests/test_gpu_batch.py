"""Batches: many instances of different sizes in one persistent launch per
kernel form, replayed as one CUDA graph, through the C ABI.

Every member of a batch must give what its own run gives: against the FP64
oracle trajectory by trajectory (common random numbers), and against an
ordinary aqt_run of the same context inputs. SIMT results do not depend on
the tile shape the autotuner picks (the rotation sums over levels in the
same order, the norms reduce over the same lanes), so final states and jumps
are compared bit for bit there; the per-grid sums over trajectories are
summed tile by tile, so they agree to rounding.
"""
import numpy as np
import pytest

import workloads as W
from test_gpu_parity import compare_crn, jumps_by_traj

pytestmark = pytest.mark.gpu


def _session(A, inst, precision, M):
    S = A.Session(inst, precision=precision, M=M)
    S.build()
    return S


def _batch(A, sessions):
    import torch
    b = A.aqt_batch_create([S.ctx for S in sessions])
    ws = torch.empty(max(A.aqt_batch_workspace_size(b), 256), dtype=torch.uint8, device="cuda:0")
    A.aqt_batch_bind_workspace(b, ws.data_ptr(), ws.numel())
    return b, ws


def _outputs(A, S):
    s1, s2 = A.aqt_get_observable_sums(S.ctx, S.K)
    jumps, dropped = S.jumps()
    return dict(s1=s1, s2=s2, jumps=jumps, dropped=dropped, final=S.final_state(basis=1))


def _run_batch(A, b, sessions):
    A.aqt_batch_run(b, sessions[0].stream())
    st, member = A.aqt_batch_sync(b, len(sessions))
    assert st == A.AQT_OK, (st, member, A.aqt_batch_last_error(b))
    return [_outputs(A, S) for S in sessions]


# (n_qubits, precision name, M, grid points, eta g^2, instance seed, t_f): uneven
# sizes, ragged M, every kernel form (the 9-qubit member keeps a short run: the
# oracle's dense 512-level frames cost ~1 s per grid point)
MIXED = [
    (6, "FP32", 40, 41, 0.02, 61, 5.0),
    (7, "F16SPLIT", 40, 41, 0.02, 71, 5.0),
    (8, "F16SPLIT", 24, 31, 0.01, 81, 5.0),
    (4, "FP64", 50, 101, 0.03, 41, 5.0),
    (9, "FP32", 9, 11, 0.05, 91, 2.0),
]
TOL = {"FP64": (1e-10, 1e-10, 1.0), "FP32": (1e-7, 1e-6, 0.97), "F16SPLIT": (1e-6, 1e-6, 0.97)}


def test_batch_mixed_sizes_against_oracle(aqt_lib):
    """n = 4 .. 9 (N = 16 .. 512) in FP64, FP32 and split FP16 in one batch:
    each member against the FP64 oracle with common random numbers; a second
    run (graph replay) repeats the first bit for bit."""
    A = aqt_lib
    insts, sessions = [], []
    for n, prec, M, grid, eta, seed, t_f in MIXED:
        inst = W.tfim_instance(n, seed, eta_g2=eta, t_f=t_f, n_grid=grid, seed=seed + 1000)
        insts.append(inst)
        sessions.append(_session(A, inst, getattr(A, "AQT_PREC_" + prec), M))
    b, ws = _batch(A, sessions)
    out = _run_batch(A, b, sessions)
    forms = [A.aqt_batch_get_shape(b, i)[0] for i in range(len(sessions))]
    assert forms == [1, 2, 2, 0, 1]
    total_jumps = 0
    for (n, prec, M, grid, eta, seed, t_f), inst, res in zip(MIXED, insts, out):
        t_tol, s_tol, frac = TOL[prec]
        assert res["dropped"] == 0
        p, oj, _ = compare_crn(inst, res, list(range(M)), t_tol=t_tol, state_tol=s_tol, min_identical=frac)
        total_jumps += len(oj)
        # per-trajectory populations agree to the state tolerance (FP64: 1e-10)
        atol = 2e-10 * M if prec == "FP64" else 2e-4 * M
        assert np.max(np.abs(res["s1"] - p.sum(axis=0))) < atol, (n, prec)
    assert total_jumps > 20
    again = _run_batch(A, b, sessions)
    for r1, r2 in zip(out, again):
        assert np.array_equal(r1["s1"], r2["s1"]) and np.array_equal(r1["final"], r2["final"])
        assert np.array_equal(r1["jumps"], r2["jumps"])
    A.aqt_batch_destroy(b)
    for S in sessions:
        S.close()


def test_batch_matches_standalone_runs(aqt_lib):
    """Members up to N = 512 against aqt_run of the same inputs."""
    A = aqt_lib
    specs = [(9, "FP32", 12, 6, 0.02, 101), (5, "FP64", 70, 61, 0.03, 51), (7, "FP32", 33, 41, 0.02, 72),
             (8, "F16SPLIT", 100, 21, 0.01, 82), (2, "FP64", 5, 11, 0.05, 21)]
    sessions, alone = [], []
    for n, prec, M, grid, eta, seed in specs:
        inst = W.tfim_instance(n, seed, eta_g2=eta, t_f=4.0, n_grid=grid, seed=seed + 7)
        pr = getattr(A, "AQT_PREC_" + prec)
        sessions.append(_session(A, inst, pr, M))
        S = _session(A, inst, pr, M)
        assert S.run() == A.AQT_OK
        alone.append(_outputs(A, S))
        S.close()
    b, ws = _batch(A, sessions)
    A.aqt_batch_tune(b, sessions[0].stream())
    out = _run_batch(A, b, sessions)
    for (n, prec, M, grid, eta, seed), r, a in zip(specs, out, alone):
        if prec == "F16SPLIT":
            # the tile shapes differ, so the tensor-core products may differ in
            # their last bits
            ga, gb = jumps_by_traj(r["jumps"]), jumps_by_traj(a["jumps"])
            same = [t for t in range(M) if [tuple(x)[:6] for x in ga.get(t, [])] == [tuple(x)[:6] for x in gb.get(t, [])]]
            assert len(same) >= 0.97 * M
            ov = np.abs(np.einsum("mi,mi->m", r["final"][same].conj(), a["final"][same]))
            assert np.max(np.abs(ov - 1.0)) < 1e-6
            assert np.max(np.abs(r["s1"] - a["s1"])) <= 1e-5 * M + (M - len(same))
        else:
            np.testing.assert_allclose(r["s1"], a["s1"], rtol=1e-12, atol=1e-12)
            assert np.array_equal(r["final"], a["final"]), (n, prec)
            assert np.array_equal(r["jumps"], a["jumps"]), (n, prec)
    shape = A.aqt_batch_get_shape(b, 0)
    assert shape[0] == 1 and shape[2] in (2, 4, 8) and shape[3] == -(-12 // shape[1])
    A.aqt_batch_destroy(b)
    for S in sessions:
        S.close()


def test_batch_refuses_a_changed_member(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(3, 5, eta_g2=0.02, t_f=2.0, n_grid=11, seed=3)
    S = _session(A, inst, A.AQT_PREC_FP64, 16)
    b, ws = _batch(A, [S])
    A.aqt_set_grid(S.ctx, 2.0, 12)
    with pytest.raises(A.AqtError) as e:
        A.aqt_batch_run(b, 0)
    assert e.value.status == A.AQT_EINVAL and "changed" in str(e.value)
    A.aqt_batch_destroy(b)
    S.close()
