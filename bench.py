"""Benchmark: trajectory-steps/s of the AME quantum-jump path on GB300.

Workload (default): 8-qubit transverse-field Ising annealing, N = 256 levels
(all kept), seeded complete-graph h, J, Ohmic bath eta g^2 = 1e-3,
omega_c = 8 pi rad/ns, T = 12.1 mK, t_f = 10 ns, 2000-point grid, M = 10^4
trajectories. One bench step = one full propagation of all M trajectories
over the whole grid (aqt_run), with the FP64 tables already resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 launch with torch.distributed.run; each rank runs M trajectories
with its own seed (weak scaling) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "trajectory-steps/s"
UNIT = "trajectory-steps/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# DRAM bytes (read + write) of one propagate_tc launch, by workload (n, N, M, n_grid, t_f), from a 1-pass
# ncu capture of the kernel as it is now (dram__bytes_read.sum + dram__bytes_write.sum); a workload not
# listed, or a kernel changed since its capture, reports null.
TC_TRAFFIC = {}

def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 60 for f16split, 3 for fp32 / fp64, 5 for the reference arm)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="main", choices=["main", "small", "batch", "grad"],
                    help="main: 8 qubits, N = 256 (default); small: 4 qubits, N = 16; batch: 64 instances of "
                         "6-8 qubits in one batched launch; grad: d<P_GS(1)>/dtheta of the 8-qubit instance with an "
                         "8-knot schedule, M = 2^14 (adjoint sweep against the forward run)")
    ap.add_argument("--batch-qubits", default="6,7,8", help="batch: qubit counts cycled over the instances")
    ap.add_argument("--batch-instances", type=int, default=64)
    ap.add_argument("--precision", default=None, choices=["f16split", "fp32", "fp64"],
                    help="default: f16split for main, fp64 for small")
    ap.add_argument("--tf", type=float, default=None, help="default: 10 ns (main, small), 20 ns (batch)")
    ap.add_argument("--M", type=int, default=None, help="default: 10^4 (main), 1000 (small)")
    ap.add_argument("--n-grid", type=int, default=None, help="default: 2000 (main), 1000 (small)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the in-process tensor / SIMT peak measurement")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=40)
    ap.add_argument("--cpu-sample-traj", type=int, default=2000)
    a = ap.parse_args()
    if a.precision is None:
        a.precision = {"small": "fp64", "grad": "fp32"}.get(a.config, "f16split")
    if a.M is None:
        a.M = {"main": 10_000, "small": 1000, "batch": 2048, "grad": 1 << 14}[a.config]
    if a.n_grid is None:
        a.n_grid = 2000 if a.config in ("main", "grad") else 1000
    if a.tf is None:
        a.tf = 20.0 if a.config == "batch" else 10.0
    return a


def workload(args):
    import workloads as W
    if args.config == "small":
        return W.cfg_small(t_f=args.tf, M=args.M, n_grid=args.n_grid)
    if args.config == "grad":
        return W.cfg_grad(t_f=args.tf, M=args.M, n_grid=args.n_grid)
    return W.cfg_main(t_f=args.tf, M=args.M, n_grid=args.n_grid)


def measure_peaks(device) -> dict:
    """Dense matrix-product rates of this GPU in TFLOP/s, measured here with
    library GEMMs (torch.matmul, CUDA events, best of 5 after warm-up): FP16
    and TF32 on the tensor cores, FP32 without TF32 and FP64. They are the
    roofline denominators of the kernels whose arithmetic they match; no clock
    or power setting is touched."""
    import torch
    out = {}
    old_tf32 = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, n, tf32 in (("fp16", torch.float16, 8192, False), ("tf32", torch.float32, 8192, True),
                                  ("fp32", torch.float32, 4096, False), ("fp64", torch.float64, 2048, False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device=device, dtype=dt)
            b = torch.randn(n, n, device=device, dtype=dt)
            for _ in range(3):
                torch.matmul(a, b)
            best = float("inf")
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name] = 2.0 * n ** 3 / best / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old_tf32
    torch.cuda.empty_cache()
    return out


def rank_seed(base: int, rank: int) -> int:
    """Trajectory-stream seed of one rank: every rank runs its own M
    trajectories (weak scaling), on its own Philox key."""
    return base + rank


def max_over_ranks(ms: float, device=None) -> float:
    """The job's timed region ends with its slowest rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks -----
REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown", 0x100: "display_clocks_setting"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while timing."""

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None
            return
        # the timed region starts only once nvidia-smi is answering (bounded wait)
        t_end = time.perf_counter() + 5.0
        while not self.lines and self.proc.poll() is None and time.perf_counter() < t_end:
            time.sleep(0.01)
        self.lines.clear()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 3:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                bits = int(parts[2], 16)
            except ValueError:
                continue
            for b, name in REASON_BITS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def alu_fp32_peak_tflops(num_sms: int, mhz: float) -> float:
    # 128 FP32 FMA lanes per SM per clock, 2 flops per FMA
    return num_sms * 128 * 2 * mhz * 1e6 / 1e12


def alu_fp64_peak_tflops(num_sms: int, mhz: float) -> float:
    # 1.25 TFLOP/s FP64 nominal on GB300 at 2070 MHz, scaled by clock
    return 1.25 * mhz / 2070.0


# ------------------------------------------------------------- CPU baseline ---
def cpu_baseline_run(args, n_traj: int, n_steps: int, first: int = 0):
    """The FP64 oracle's trajectory propagation on a bounded sample of the
    workload: trajectories first .. first + n_traj - 1 over the first n_steps
    grid steps. The per-grid eigensystem/propagator setup is excluded, as the
    GPU's FP64 table build is excluded from its number. Single thread."""
    from oracle import ame, trajectories
    inst = workload(args)
    _, dt = __import__("oracle.model", fromlist=["grid"]).grid(inst)
    tau = 0.5 * dt
    prop_time = 0.0
    trajs = None
    prev = None
    for k, fr in enumerate(ame.frames(inst)):
        if k > n_steps:
            break
        piece = trajectories.Piece(fr, tau)
        if k == 0:
            trajs = [trajectories.Trajectory(t, inst.seed, fr.eig.V[:, 0]) for t in range(first, first + n_traj)]
        else:
            t0 = time.perf_counter()
            for tr in trajs:
                tr.advance(prev, tau, (k - 1) * dt, k - 1, 1)
                tr.advance(piece, tau, (k - 1) * dt + tau, k, 0)
            prop_time += time.perf_counter() - t0
        prev = piece
    return n_traj * n_steps / prop_time, prop_time


def cpu_baseline(args, n_traj=None, n_steps=None):
    """Run the oracle leg in a single-threaded child process."""
    n_traj = n_traj or args.cpu_sample_traj
    n_steps = n_steps or args.cpu_sample_steps
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "a = bench.parse_from(%r); v, t = bench.cpu_baseline_run(a, %d, %d); "
            "print(json.dumps({'value': v, 'seconds': t}))") % (ROOT, sys.argv[1:], n_traj, n_steps)
    r = subprocess.run([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                       text=True, timeout=1800)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-500:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n_traj} trajectories x first {n_steps} grid steps of the same workload, FP64 "
                      f"numpy/scipy, propagation only ({d['seconds']:.1f} s)"}


def _cpu_worker(job):
    argv, first, n_traj, n_steps = job
    v, t = cpu_baseline_run(parse_from(argv), n_traj, n_steps, first)
    return v, t


def cpu_baseline_all_cores(args, n_traj=None, n_steps=None):
    """The same oracle leg on every host core: one single-threaded worker per
    core (spawned processes), each on its own trajectories; the rate is the
    sum of the workers' rates while they all run."""
    import multiprocessing
    n_traj = n_traj or args.cpu_sample_traj
    n_steps = n_steps or args.cpu_sample_steps
    cores = len(os.sched_getaffinity(0))
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    jobs = [(sys.argv[1:], i * n_traj, n_traj, n_steps) for i in range(cores)]
    try:
        with multiprocessing.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_cpu_worker, jobs)
    except Exception as e:  # noqa: BLE001
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "error": str(e)[:300]}
    return {"value": sum(v for v, _ in res), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} workers x {n_traj} trajectories x first {n_steps} grid steps of the same workload, "
                      f"FP64 numpy/scipy, propagation only ({max(t for _, t in res):.1f} s)"}


def parse_from(argv):
    old = sys.argv
    sys.argv = [old[0]] + list(argv)
    try:
        return parse()
    finally:
        sys.argv = old


# ------------------------------------------------------------------ ours ------
def run_ours(args):
    import numpy as np
    import torch

    from paper_1710_03431_gb300 import aqt as A

    rank, world, local = dist_env()
    if args.steps is None:  # a timed region of about a second
        args.steps = {"f16split": 60, "fp32": 3, "fp64": 3}[args.precision]
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    inst = workload(args)
    prec = {"fp32": A.AQT_PREC_FP32, "fp64": A.AQT_PREC_FP64, "f16split": A.AQT_PREC_F16SPLIT}[args.precision]
    seed = rank_seed(inst.seed, rank)
    sess = A.Session(inst, precision=prec, device=local, seed=seed)
    t0 = time.perf_counter()
    sess.build()
    torch.cuda.synchronize()
    table_s = time.perf_counter() - t0

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        sess.run()
    # timed region
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    per = []
    ev0.record(stream)
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        A.aqt_run(sess.ctx, stream.cuda_stream)
        b.record(stream)
        per.append((a, b))
    ev1.record(stream)
    torch.cuda.synchronize()
    status = A.aqt_sync(sess.ctx)
    ck = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    kern_ms = [a.elapsed_time(b) for a, b in per]
    if world > 1:
        elapsed_ms = max_over_ranks(elapsed_ms, dev)
    ms_per_step = elapsed_ms / args.steps
    N, M, K = 1 << inst.n_qubits, sess.M, inst.n_grid
    traj_steps = M * (K - 1)
    value = world * traj_steps / (ms_per_step / 1e3)
    mean, se = sess.observables()
    jumps, dropped = sess.jumps()

    # e2e: the public C ABI with host buffers, tables built inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        ctx2 = A.aqt_create(local)
        ws = sess.ws
        h2d = 0
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(args.e2e_steps):
            A.aqt_set_ising(ctx2, inst.n_qubits, inst.hz, inst.J)
            A.aqt_set_schedule(ctx2, inst.sched_s, inst.sched_A, inst.sched_B)
            A.aqt_set_bath(ctx2, inst.eta_g2, inst.omega_c, inst.beta, inst.lamb_shift)
            A.aqt_set_grid(ctx2, inst.t_f, inst.n_grid)
            A.aqt_set_trajectories(ctx2, M, seed, prec, A.AQT_JUMP_REFINED, sess.jcap)
            A.aqt_bind_workspace(ctx2, ws.data_ptr(), ws.numel())
            A.aqt_build_tables(ctx2, stream.cuda_stream)
            A.aqt_run(ctx2, stream.cuda_stream)
            A.aqt_sync(ctx2)
            m2, s2 = A.aqt_get_observables(ctx2, K)
        e2e_s = (time.perf_counter() - t1) / args.e2e_steps
        # bytes aqt_build_tables copied to the device (as the library counts them)
        h2d = int(A.aqt_debug_table(ctx2, 8, 0, (2,))[1])
        A.aqt_destroy(ctx2)
        e2e = {"value": world * traj_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(K * 2 * 8 + 12), "seconds_per_step": e2e_s,
               "includes": "set_* + FP64 host table build + H2D + run + sync + observables D2H"}

    if rank != 0:
        return
    props = torch.cuda.get_device_properties(local)
    num_sms = props.multi_processor_count
    kern_avg_s = statistics.mean(kern_ms) / 1e3
    flops = 4.0 * N * N * traj_steps
    mhz = ck.get("sm_max_mhz") or 2070.0
    achieved = flops / kern_avg_s / 1e12
    peaks, src = measured_peaks()
    here = {} if args.no_peaks else measure_peaks(dev)
    if prec == A.AQT_PREC_F16SPLIT:
        if "fp16" in here:
            peak = here["fp16"]
            peak_src = "dense fp16 tensor rate measured in this process (cuBLAS 8192^3, best of 5, burst)"
        else:
            peak = float(peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"]))
            peak_src = f"dense bf16 tensor peak, burst, {src} (MEASURED_PEAKS.json bf16_tflops; fp16 taken at the bf16 rate)"
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TC_TRAFFIC.get((inst.n_qubits, N, M, K, float(inst.t_f))), "kernel": "propagate_tc",
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "algorithmic": "4 N^2 flop per trajectory-step (real N x N rotation of a complex state); "
                               "the split form issues 3x that on the FP16 tensor pipe",
                "issued_mma_frac": 3.0 * achieved / peak, "peak_source": peak_src,
                "bf16_measured_peaks_json": peaks.get("bf16_tflops")}
    else:
        key = "fp32" if prec == A.AQT_PREC_FP32 else "fp64"
        if key in here:
            peak = here[key]
            peak_src = f"dense {key} matrix-product rate measured in this process (cuBLAS, no TF32, best of 5)"
        elif prec == A.AQT_PREC_FP32:
            peak = alu_fp32_peak_tflops(num_sms, mhz)
            peak_src = f"FP32 FMA: {num_sms} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz (nominal)"
        else:
            peak = alu_fp64_peak_tflops(num_sms, mhz)
            peak_src = f"FP64: 1.25 TFLOP/s nominal scaled to {mhz:.0f} MHz"
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": f"propagate_simt<{'float' if prec else 'double'}>",
                "algorithmic": "4 N^2 flop per trajectory-step (real N x N rotation of a complex state)",
                "peak_source": peak_src}
    roof["peaks_measured_here_tflops"] = here
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        one = cpu_baseline(args)
        cpu = cpu_baseline_all_cores(args)
        cpu["one_core"] = one
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {A.AQT_PREC_FP32: "f32", A.AQT_PREC_FP64: "f64",
                                       A.AQT_PREC_F16SPLIT: "f16x3-f32acc"}[prec], "data": "synthetic",
        "config": {"workload": f"tfim-{inst.n_qubits}q-N{N}-M{M}-grid{K}-tf{inst.t_f:g}ns",
                   "N": N, "M": M, "n_grid": K, "t_f_ns": inst.t_f, "precision": args.precision,
                   "tables": "FP64 eigensystems, rates, jump tables; rotation tables in the state precision",
                   "l2": f"rotation tables {((K - 1) * N * N * (8 if prec == A.AQT_PREC_FP64 else 4)) / 1e9:.2f} GB"
                         " > L2, streamed once per run",
                   "parallelism": f"trajectories x{world}"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * args.steps, "clocks": ck,
        "table_build_s": table_s, "status": A.STATUS_NAMES.get(status, status),
        "gs_population_final": {"mean": float(mean[-1]), "stderr": float(se[-1])},
        "jumps_per_trajectory": (len(jumps) + dropped) / M,
    }
    print(json.dumps(line))


# ------------------------------------------------------------- reference ------
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    if args.steps is None:
        args.steps = 5
    vals = []
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state beyond imports
    d = None
    for _ in range(args.steps):
        d = cpu_baseline(args, n_traj=max(8, args.cpu_sample_traj // 4), n_steps=max(5, args.cpu_sample_steps // 4))
        if d["value"] is None:
            print(json.dumps({"impl": "reference", "unavailable": "oracle leg failed: " + d.get("error", "")[:200]}))
            return
        vals.append(d["value"])
    v = statistics.mean(vals)
    inst = workload(args)
    N = 1 << inst.n_qubits
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"tfim-{inst.n_qubits}q-N{N}-M{inst.M}-grid{inst.n_grid}-tf{inst.t_f:g}ns",
                   "N": N, "M": inst.M, "n_grid": inst.n_grid, "t_f_ns": inst.t_f},
        "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": 1, "sample": d["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ batch -----
def run_batch(args):
    """Many instances of uneven size in one batch (aqt_batch_run: one CUDA
    graph with one persistent launch per kernel form). precision f16split:
    members with N = 128 / 256 on the tensor cores, the others SIMT FP32;
    fp32 / fp64: every member SIMT in that precision. One bench step = one
    run of every member over its whole grid."""
    import torch

    import workloads as W
    from paper_1710_03431_gb300 import aqt as A

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if args.steps is None:
        args.steps = 5
    qubits = tuple(int(x) for x in args.batch_qubits.split(","))
    insts = W.cfg_batch(n_instances=args.batch_instances, qubits=qubits, M=args.M, n_grid=args.n_grid, t_f=args.tf)
    sessions = []
    t0 = time.perf_counter()
    for inst in insts:
        N = 1 << inst.n_qubits
        if args.precision == "f16split":
            prec = A.AQT_PREC_F16SPLIT if N in (128, 256) else A.AQT_PREC_FP32
        else:
            prec = {"fp32": A.AQT_PREC_FP32, "fp64": A.AQT_PREC_FP64}[args.precision]
        S = A.Session(inst, precision=prec, device=local, seed=rank_seed(inst.seed, rank))
        S.build()
        sessions.append(S)
    torch.cuda.synchronize()
    table_s = time.perf_counter() - t0
    b = A.aqt_batch_create([S.ctx for S in sessions])
    ws = torch.empty(A.aqt_batch_workspace_size(b), dtype=torch.uint8, device=f"cuda:{local}")
    A.aqt_batch_bind_workspace(b, ws.data_ptr(), ws.numel())
    stream = torch.cuda.current_stream()
    t1 = time.perf_counter()
    A.aqt_batch_tune(b, stream.cuda_stream)
    tune_s = time.perf_counter() - t1
    for _ in range(args.warmup):
        A.aqt_batch_run(b, stream.cuda_stream)
        A.aqt_batch_sync(b, len(sessions))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        A.aqt_batch_run(b, stream.cuda_stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    st, member = A.aqt_batch_sync(b, len(sessions))
    ck = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    if world > 1:
        elapsed_ms = max_over_ranks(elapsed_ms, torch.device(f"cuda:{local}"))
    ms_per_step = elapsed_ms / args.steps
    traj_steps = sum(S.M * (S.K - 1) for S in sessions)
    flops = sum(4.0 * S.N * S.N * S.M * (S.K - 1) for S in sessions)
    shapes = [A.aqt_batch_get_shape(b, i) for i in range(len(sessions))]
    if rank != 0:
        return
    forms = {}
    for S, sh in zip(sessions, shapes):
        key = ["simt-fp64", "simt-fp32", "tensor-f16x3"][sh[0]] + f"-N{S.N}"
        f = forms.setdefault(key, {"instances": 0, "tt": sh[1], "ra_or_mh": sh[2], "tiles": 0})
        f["instances"] += 1
        f["tiles"] += sh[3]
    achieved = flops / (ms_per_step / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": world * traj_steps / (ms_per_step / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f16split": "f16x3-f32acc+f32", "fp32": "f32", "fp64": "f64"}[args.precision], "data": "synthetic",
        "config": {"workload": f"tfim-batch-{len(insts)}x{'/'.join(map(str, qubits))}q-M{insts[0].M}-"
                               f"grid{insts[0].n_grid}-tf{insts[0].t_f:g}ns",
                   "instances": len(insts), "qubits": list(qubits), "M_each": insts[0].M,
                   "n_grid": insts[0].n_grid, "t_f_ns": insts[0].t_f, "precision": args.precision,
                   "launch": "one CUDA graph per run: counter resets, one persistent kernel per form, reduction",
                   "forms": forms},
        "roofline": {"bound": "mixed", "achieved": achieved, "unit": "TFLOP/s",
                     "algorithmic": "4 N^2 flop per trajectory-step summed over the members"},
        "status": A.STATUS_NAMES.get(st, st), "clocks": ck, "table_build_s": table_s, "tune_s": tune_s,
        "gpu_launches": args.steps * (1 + len(forms)),
    }
    print(json.dumps(line))
    A.aqt_batch_destroy(b)
    for S in sessions:
        S.close()


# ------------------------------------------------------------------- grad -----
def run_grad(args):
    """Gradient of <P_GS(1)> in the 2 x 8 schedule control values, 8 fields and
    28 couplings (SIMT FP32 or FP64). One step = the checkpointed forward run
    plus the adjoint sweep (device), timed with CUDA events; the plain forward
    run (aqt_run) of the same trajectories is timed beside it, and the host's
    FP64 contraction (aqt_grad_get) separately with the wall clock."""
    import torch

    from paper_1710_03431_gb300 import aqt as A

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if args.steps is None:
        args.steps = 3
    inst = workload(args)
    prec = {"fp32": A.AQT_PREC_FP32, "fp64": A.AQT_PREC_FP64}[args.precision]
    S = A.Session(inst, precision=prec, device=local, seed=rank_seed(inst.seed, rank))
    t0 = time.perf_counter()
    S.build()
    table_s = time.perf_counter() - t0
    S.grad_allocate(64)
    stream = torch.cuda.current_stream()
    P = A.aqt_grad_n_params(S.ctx)

    def fwd():
        A.aqt_run(S.ctx, stream.cuda_stream)

    def grad_device():
        A.aqt_grad_forward(S.ctx, stream.cuda_stream)
        A.aqt_grad_backward(S.ctx, float("nan"), stream.cuda_stream)

    for _ in range(args.warmup):
        fwd()
        grad_device()
        A.aqt_grad_get(S.ctx, P)
    torch.cuda.synchronize()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    fwd_ms = timed(fwd)
    grad_ms = timed(grad_device)
    ck = clocks.stop()
    t1 = time.perf_counter()
    g, value = A.aqt_grad_get(S.ctx, P)
    host_s = time.perf_counter() - t1
    if world > 1:
        grad_ms = max_over_ranks(grad_ms, torch.device(f"cuda:{local}"))
        fwd_ms = max_over_ranks(fwd_ms, torch.device(f"cuda:{local}"))
    K, M = inst.n_grid, S.M
    traj_steps = M * (K - 1)
    S.close()
    if rank != 0:
        return
    line = {
        "metric": "gradient trajectory-steps/s (checkpointed forward + adjoint sweep)",
        "value": world * traj_steps / (grad_ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": grad_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {A.AQT_PREC_FP32: "f32", A.AQT_PREC_FP64: "f64"}[prec], "data": "synthetic",
        "config": {"workload": f"tfim-8q-N256-M{M}-grid{K}-tf{inst.t_f:g}ns-{len(inst.sched_s)}knots-grad",
                   "N": 1 << inst.n_qubits, "M": M, "n_grid": K, "params": P, "checkpoint_every": 64,
                   "precision": args.precision, "parallelism": f"trajectories x{world}"},
        "forward_ms": fwd_ms, "grad_over_forward": grad_ms / fwd_ms,
        "host_contraction_s": host_s,
        "grad_plus_host_over_forward": (grad_ms / 1e3 + host_s) / (fwd_ms / 1e3),
        "p_gs_final": value, "grad_norm": float(np.sqrt(np.nansum(np.asarray(g) ** 2))),
        "undefined_params": int(np.isnan(g).sum()),
        "clocks": ck, "table_build_s": table_s, "gpu_launches": args.steps * (2 + 2 + 3 * ((K + 63) // 64)),
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batch":
        run_batch(args)
    elif args.config == "grad":
        run_grad(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
