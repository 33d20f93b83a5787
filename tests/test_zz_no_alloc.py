"""The static-scratch run entry point against the ordinary run.

aqt_run_static_scratch is for callers that cannot allocate device memory
when they run (a fixed memory pool, or threads where allocation is not
allowed): its scratch lives in an array compiled into the library. This test
allocates the output buffers itself (the caller's job), calls the entry point
twice in a row through the C ABI and compares both results with aqt_run on
the same context. It lives in its own file so that it is collected last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,M,grid,precision", [(3, 300, 201, 0), (7, 64, 101, 2)])
def test_static_scratch_matches_ordinary_run(aqt_lib, n, M, grid, precision):
    """FP64 SIMT path (jump vectors in the static array) and tensor-core path
    (jump vectors and per-trajectory patch products in the static array)."""
    import torch

    A = aqt_lib
    inst = W.tfim_instance(n, 44 + n, eta_g2=0.02, t_f=6.0, n_grid=grid, seed=3)
    S = A.Session(inst, precision=precision, M=M)
    S.build()
    assert S.run() == A.AQT_OK
    ref_s1, ref_s2 = A.aqt_get_observable_sums(S.ctx, inst.n_grid)
    ref_final = A.aqt_get_final_state(S.ctx, 0, M, S.N)
    ref_jumps, _ = S.jumps()

    dev = torch.device("cuda:0")
    obs = torch.empty((inst.n_grid, 2), dtype=torch.float64, device=dev)
    fin = torch.empty((M, S.N, 2), dtype=torch.float64, device=dev)
    cap = 4 * len(ref_jumps) + 16
    jrec = torch.empty((cap * A.JUMP_DTYPE.itemsize,), dtype=torch.uint8, device=dev)
    cnt = torch.empty((1,), dtype=torch.int64, device=dev)
    status = torch.empty((1,), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    for call in range(2):
        obs.fill_(-1.0)
        fin.fill_(-1.0)
        A.aqt_run_static_scratch(S.ctx, stream.cuda_stream, obs.data_ptr(), fin.data_ptr(), jrec.data_ptr(), cap,
                                 cnt.data_ptr(), status.data_ptr())
        torch.cuda.synchronize()
        assert int(status.item()) == 0, call
        n = int(cnt.item())
        assert n == len(ref_jumps), (call, n, len(ref_jumps))
        o = obs.cpu().numpy()
        np.testing.assert_array_equal(o[:, 0], ref_s1)
        np.testing.assert_array_equal(o[:, 1], ref_s2)
        f = fin.cpu().numpy()
        np.testing.assert_array_equal(f[..., 0] + 1j * f[..., 1], ref_final)
        recs = np.frombuffer(jrec.cpu().numpy().tobytes()[: n * A.JUMP_DTYPE.itemsize], dtype=A.JUMP_DTYPE)
        got = sorted((int(r["traj"]), float(r["t"]), int(r["src"]), int(r["dst"])) for r in recs)
        exp = sorted((int(r["traj"]), float(r["t"]), int(r["src"]), int(r["dst"])) for r in ref_jumps)
        assert [g[0::2] + (g[3],) for g in got] == [e[0::2] + (e[3],) for e in exp]
        assert all(g[1] == e[1] for g, e in zip(got, exp))
    S.close()


def test_static_scratch_rejects_oversized_runs(aqt_lib):
    A = aqt_lib
    inst = W.tfim_instance(6, 5, n_grid=4000)
    c = A.aqt_create(0)
    A.aqt_set_ising(c, inst.n_qubits, inst.hz, inst.J)
    A.aqt_set_schedule(c, inst.sched_s, inst.sched_A, inst.sched_B)
    A.aqt_set_bath(c, inst.eta_g2, inst.omega_c, inst.beta, inst.lamb_shift)
    A.aqt_set_grid(c, inst.t_f, inst.n_grid)
    A.aqt_set_trajectories(c, 200_000, 1, A.AQT_PREC_FP64, 0, 16)
    with pytest.raises(A.AqtError) as e:
        A.aqt_run_static_scratch(c, 0, 1 << 20, 1 << 20, 1 << 20, 16, 1 << 20, 1 << 20)
    assert e.value.status == A.AQT_EINVAL and "static array" in str(e.value)
    A.aqt_destroy(c)
