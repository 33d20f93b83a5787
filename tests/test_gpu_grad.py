"""Gradient runs (aqt_grad_*) against the gradient oracle, through the C ABI.

* FP64, common random numbers: the device's gradient is the mean over its
  trajectories of the record-fixed estimate; the oracle replays the same
  records (same jumps, checked) at theta +- delta and differences them. The
  two must agree to the FD's accuracy, element by element, with several
  checkpoint segments and a ragged last one.
* The field-scaling identity of the Hamiltonian family (exact per trajectory).
* The mean over many trajectories against central differences of the
  density-matrix AME (unbiasedness; statistical tolerance).
* FP32 against FP64 on the same streams, and the torch.autograd.Function.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import gradient as G
from oracle import trajectories

pytestmark = pytest.mark.gpu


def hot(n=3, seed=5, K=30, t_f=4.0, eta=0.04, M=48):
    return W.tfim_instance(n, seed, eta_g2=eta, t_f=t_f, n_grid=K, seed=11, M=M)


def device_grad(A, inst, precision, baseline, every, M=None, seed=None):
    S = A.Session(inst, precision=precision, M=M, seed=seed)
    S.build()
    g, v = S.gradient(baseline=baseline, checkpoint_every=every)
    jumps, dropped = S.jumps()
    S.close()
    assert dropped == 0
    return g, v, jumps


@pytest.mark.parametrize("every", [7, 64])
def test_fp64_gradient_matches_record_replay(aqt_lib, every):
    A = aqt_lib
    inst = hot()
    b = 0.55
    g, v, jumps = device_grad(A, inst, A.AQT_PREC_FP64, b, every)
    M = inst.M
    p, ojumps, _ = trajectories.sample(inst, list(range(M)))
    assert len(jumps) == len(ojumps) > 10
    for x, y in zip(sorted(jumps.tolist(), key=lambda r: (r[0], r[6])),
                    sorted(ojumps, key=lambda r: (r["traj"], r["t"]))):
        assert (x[0], x[1], x[2], x[3], x[4], x[5]) == (y["traj"], y["grid"], y["half"], y["alpha"], y["src"], y["dst"])
    assert abs(v - p[:, -1].mean()) < 1e-9
    by = {t: [] for t in range(M)}
    for j in ojumps:
        by[j["traj"]].append(j)
    ref = np.mean([G.trajectory_gradient_fd(inst, by[t], baseline=b)[0] for t in range(M)], axis=0)
    und = G.undefined_params(inst)
    assert np.array_equal(np.isnan(g), und), (g, und)
    scale = np.max(np.abs(ref[~und]))
    assert scale > 1e-3
    np.testing.assert_allclose(g[~und], ref[~und], rtol=1e-6, atol=1e-7 * scale)


def test_tiled_outer_products_identity_and_segments(aqt_lib):
    """N = 128: the outer products run on the tiled kernel (128 x 128 tiles,
    trajectories split over blocks and added in FP64). The field-scaling
    identity holds per trajectory, so the sum over trajectories checks the
    tiled sums through every parameter class; two checkpoint spacings give
    the same gradient to rounding."""
    A = aqt_lib
    inst = W.tfim_instance(7, 3, eta_g2=0.05, t_f=2.0, n_grid=40, seed=5, M=2100)
    g1, _, j1 = device_grad(A, inst, A.AQT_PREC_FP64, 0.5, 7)
    g2, _, j2 = device_grad(A, inst, A.AQT_PREC_FP64, 0.5, 64)
    assert len(j1) == len(j2) > 100
    th = G.param_vector(inst)
    k = len(inst.sched_s)
    for g in (g1, g2):
        lhs = np.dot(th[2 * k:], g[2 * k:])
        rhs = np.nansum(th[k:2 * k] * np.where(np.isnan(g[k:2 * k]), 0.0, g[k:2 * k]))
        assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs)), (lhs, rhs)
    ok = ~np.isnan(g1)
    assert np.array_equal(ok, ~np.isnan(g2))
    np.testing.assert_allclose(g1[ok], g2[ok], rtol=1e-9, atol=1e-12 * np.max(np.abs(g1[ok])))
    # the FP32 form of the tiled kernel (state-precision sums over blocks of 2048 trajectories)
    g32, _, j32 = device_grad(A, inst, A.AQT_PREC_FP32, 0.5, 16)
    scale = np.max(np.abs(g1[ok]))
    tol = (2e-4 if len(j32) == len(j1) else 2e-2) * scale
    assert np.max(np.abs(g32[ok] - g1[ok])) <= tol, (g32, g1)


def test_field_scaling_identity_on_device(aqt_lib):
    A = aqt_lib
    inst = hot(n=4, seed=9, K=50, M=256)
    g, _, _ = device_grad(A, inst, A.AQT_PREC_FP64, float("nan"), 16)
    th = G.param_vector(inst)
    k = len(inst.sched_s)
    lhs = np.dot(th[2 * k:], g[2 * k:])
    rhs = np.nansum(th[k:2 * k] * np.where(np.isnan(g[k:2 * k]), 0.0, g[k:2 * k]))
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs)), (lhs, rhs)


def test_fp32_gradient_near_fp64(aqt_lib):
    A = aqt_lib
    inst = hot(n=4, seed=9, K=50, M=512)
    g64, v64, j64 = device_grad(A, inst, A.AQT_PREC_FP64, 0.6, 16)
    g32, v32, j32 = device_grad(A, inst, A.AQT_PREC_FP32, 0.6, 16)
    ok = ~np.isnan(g64)
    assert np.array_equal(ok, ~np.isnan(g32))
    # a trajectory whose FP32 jump sequence leaves the FP64 one changes its own
    # estimate by O(1) / M; otherwise the two differ by FP32 rounding
    same = len(j64) == len(j32)
    scale = np.max(np.abs(g64[ok]))
    tol = (2e-4 if same else 2e-2) * scale
    assert np.max(np.abs(g32[ok] - g64[ok])) <= tol, (g32, g64)
    assert abs(v32 - v64) < 1e-2


def test_gradient_mean_matches_density_matrix(aqt_lib):
    """Unbiasedness: four independent runs (disjoint streams) of 4096
    trajectories each against the AME's central differences."""
    A = aqt_lib
    inst = hot(n=3, seed=5, K=40, t_f=5.0, eta=0.03, M=4096)
    runs = []
    for r in range(4):
        g, _, _ = device_grad(A, inst, A.AQT_PREC_FP64, float("nan"), 64, seed=1000 + r)
        runs.append(g)
    runs = np.array(runs)
    fd = G.ame_gradient_fd(inst, delta=1e-4)
    und = G.undefined_params(inst)
    assert np.array_equal(np.isnan(runs[0]), und)
    m = runs[:, ~und].mean(axis=0)
    se = runs[:, ~und].std(axis=0, ddof=1) / 2.0
    ref = fd[~und]
    scale = np.max(np.abs(ref))
    err = np.abs(m - ref)
    assert np.all(err <= 5.0 * se + 0.02 * scale), (m, ref, se)
    # and the gradient is resolved: the largest entries are many standard errors from zero
    assert np.max(np.abs(ref) / np.maximum(se, 1e-12)) > 10


def test_autograd_function(aqt_lib):
    torch = pytest.importorskip("torch")
    from paper_1710_03431_gb300 import autograd as AG
    A = aqt_lib
    inst = hot(n=3, seed=5, K=30, M=256)
    theta = torch.tensor(AG.parameters_of(inst), dtype=torch.float64, requires_grad=True)
    y = AG.ground_population(theta, inst, precision=A.AQT_PREC_FP32, checkpoint_every=8, baseline=0.5)
    y.backward()
    g, v, _ = device_grad(A, inst, A.AQT_PREC_FP32, 0.5, 8)
    assert float(y.detach()) == v
    got = theta.grad.numpy()
    assert np.array_equal(np.isnan(got), np.isnan(g))
    ok = ~np.isnan(g)
    # the per-level sums are atomics (FP32 within a CTA, FP64 across CTAs) whose
    # order is not fixed: equal to FP32 rounding
    np.testing.assert_allclose(got[ok], g[ok], rtol=1e-5, atol=1e-9)
