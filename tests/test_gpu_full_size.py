"""The bench workload at full size (8 qubits, N = 256, M = 10^4 trajectories,
2000-point grid, t_f = 10 and 100 ns) on the tensor-core path, in the launch
configuration bench.py times.

Checks against stored oracle outputs (tests/golden, written by the committed
scripts there, which call only the oracle): sampled trajectories jump by jump,
and the trajectory mean against the FP64 density-matrix AME. Plus properties
that hold at any size: status, normalisation, record validity, determinism.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from test_gpu_parity import run_lib, se_bound

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_curve(tf):
    path = os.path.join(GOLDEN, f"cfg_main_tf{tf:g}_pgs.txt")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    return np.loadtxt(path)


@pytest.fixture(scope="module")
def full_tf10(aqt_lib):
    inst = W.cfg_main(t_f=10.0)
    return inst, run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_F16SPLIT)


def test_full_size_properties(aqt_lib, full_tf10):
    inst, res = full_tf10
    assert res["status"] == aqt_lib.AQT_OK and res["dropped"] == 0
    assert np.all(res["mean"] >= -1e-6) and np.all(res["mean"] <= 1 + 1e-6)
    nrm = np.sum(np.abs(res["final"]) ** 2, axis=1)
    assert np.max(np.abs(nrm - 1.0)) < 1e-4
    j = res["jumps"]
    assert np.all((j["t"] >= 0) & (j["t"] <= inst.t_f + 1e-9))
    assert np.all((j["src"] >= 0) & (j["src"] < 256) & (j["dst"] >= 0) & (j["dst"] < 256))
    assert np.all((j["alpha"] >= 0) & (j["alpha"] < 8))
    for t in np.unique(j["traj"])[:200]:
        tt = j["t"][j["traj"] == t]
        assert np.all(np.diff(tt) >= 0)
    # jumps between distinct levels carry a Bohr frequency of the right sign
    relax = j[(j["src"] > j["dst"])]
    assert np.all(relax["omega"] > 0)
    # P12 on the kernel's own arithmetic at full size: relative norm change of
    # one split-FP16 rotation, over all trajectories and steps (budget 1e-5)
    assert 0.0 < res["roterr"] < 1e-5


def test_full_size_samples_match_oracle(aqt_lib, full_tf10):
    path = os.path.join(GOLDEN, "cfg_main_tf10_traj.json")
    if not os.path.exists(path):
        pytest.skip("oracle samples not generated")
    gold = json.load(open(path))
    inst, res = full_tf10
    assert gold["seed"] == inst.seed and gold["n_grid"] == inst.n_grid
    recs = res["jumps"]
    same = 0
    for tr in gold["samples"]:
        g = [(int(r["grid"]), int(r["half"]), int(r["alpha"]), int(r["src"]), int(r["dst"]), float(r["t"]))
             for r in recs[recs["traj"] == tr]]
        o = [(r["grid"], r["half"], r["alpha"], r["src"], r["dst"], r["t"]) for r in gold["jumps"] if r["traj"] == tr]
        if len(g) == len(o) and all(a[:5] == b[:5] and abs(a[5] - b[5]) < 1e-5 for a, b in zip(g, o)):
            same += 1
            # final ground-manifold population (ground state of H_S(1) is level 0)
            p_gpu = abs(res["final"][tr] @ _ground_vector(aqt_lib, inst)) ** 2
            assert abs(p_gpu - gold["p_gs_every_100"][str(tr)][-1]) < 1e-4
    assert same >= len(gold["samples"]) - 1, (same, len(gold["samples"]))


_GV = {}


def _ground_vector(aqt_lib, inst):
    key = id(inst)
    if key not in _GV:
        c = aqt_lib.aqt_create(-1)
        aqt_lib.aqt_set_ising(c, inst.n_qubits, inst.hz, inst.J)
        aqt_lib.aqt_set_schedule(c, inst.sched_s, inst.sched_A, inst.sched_B)
        aqt_lib.aqt_set_bath(c, inst.eta_g2, inst.omega_c, inst.beta, inst.lamb_shift)
        aqt_lib.aqt_set_grid(c, inst.t_f, 2)
        aqt_lib.aqt_set_trajectories(c, 1, 1, 0, 0, 1)
        aqt_lib.aqt_build_tables(c, 0)
        V = aqt_lib.aqt_debug_table(c, 5, 1, (256, 256))
        aqt_lib.aqt_destroy(c)
        _GV[key] = V[:, 0].conj()
    return _GV[key]


def test_full_size_mean_matches_ame_tf10(aqt_lib, full_tf10):
    ref = _load_curve(10.0)
    inst, res = full_tf10
    for k in (250, 500, 750, 1000, 1250, 1500, 1750, 1999):
        tol = 4.0 * max(res["se"][k], se_bound(ref[k], inst.M))
        assert abs(res["mean"][k] - ref[k]) < tol, (k, res["mean"][k], ref[k], tol)


def test_full_size_mean_matches_ame_tf100(aqt_lib):
    ref = _load_curve(100.0)
    inst = W.cfg_main(t_f=100.0)
    res = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_F16SPLIT)
    assert res["status"] == aqt_lib.AQT_OK
    for k in (250, 500, 750, 1000, 1250, 1500, 1750, 1999):
        tol = 4.0 * max(res["se"][k], se_bound(ref[k], inst.M))
        assert abs(res["mean"][k] - ref[k]) < tol, (k, res["mean"][k], ref[k], tol)


def test_full_size_deterministic(aqt_lib, full_tf10):
    inst, res = full_tf10
    again = run_lib(aqt_lib, inst, aqt_lib.AQT_PREC_F16SPLIT)
    assert np.array_equal(again["s1"], res["s1"]) and np.array_equal(again["s2"], res["s2"])
    assert len(again["jumps"]) == len(res["jumps"])
