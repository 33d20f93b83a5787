"""ctypes binding of libaqt.so: the C ABI of include/aqt.h under the same names.

Argument marshalling only; every computation runs in the library. The
``Session`` helper adds what PyTorch is here for: a device workspace tensor
and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaqt.so")

AQT_OK, AQT_EINVAL, AQT_ECUDA, AQT_ENOMEM, AQT_EOVERFLOW, AQT_ENUMERIC, AQT_ENOCONV, AQT_EDEGEN, AQT_ENODEV, AQT_ETIMEOUT, \
    AQT_WDT = range(11)
AQT_PREC_FP64, AQT_PREC_FP32, AQT_PREC_F16SPLIT = 0, 1, 2
AQT_JUMP_REFINED, AQT_JUMP_GRID, AQT_JUMP_FIXED_STEP = 0, 1, 2
STATUS_NAMES = {0: "AQT_OK", 1: "AQT_EINVAL", 2: "AQT_ECUDA", 3: "AQT_ENOMEM", 4: "AQT_EOVERFLOW",
                5: "AQT_ENUMERIC", 6: "AQT_ENOCONV", 7: "AQT_EDEGEN", 8: "AQT_ENODEV", 9: "AQT_ETIMEOUT",
                10: "AQT_WDT"}

EXPORTS = ["aqt_create", "aqt_destroy", "aqt_last_error", "aqt_set_ising", "aqt_set_schedule",
           "aqt_set_bath", "aqt_set_levels", "aqt_set_grid", "aqt_set_trajectories", "aqt_workspace_size",
           "aqt_bind_workspace", "aqt_build_tables", "aqt_get_dt_bounds", "aqt_set_wait_limit", "aqt_run", "aqt_sync", "aqt_get_observables",
           "aqt_get_observable_sums", "aqt_observables_from_sums", "aqt_get_rotation_error", "aqt_get_leakage", "aqt_get_jumps", "aqt_get_final_state", "aqt_debug_table",
           "aqt_run_static_scratch", "aqt_batch_create", "aqt_batch_destroy", "aqt_batch_last_error",
           "aqt_batch_workspace_size", "aqt_batch_bind_workspace", "aqt_batch_tune", "aqt_batch_run", "aqt_batch_sync",
           "aqt_batch_get_shape", "aqt_grad_n_params", "aqt_grad_workspace_size", "aqt_grad_bind_workspace",
           "aqt_grad_forward", "aqt_grad_backward", "aqt_grad_get"]


class aqt_jump(C.Structure):
    _fields_ = [("traj", C.c_int32), ("grid", C.c_int32), ("half", C.c_int32), ("alpha", C.c_int32),
                ("src", C.c_int32), ("dst", C.c_int32), ("t", C.c_double), ("omega", C.c_double)]


JUMP_DTYPE = np.dtype([("traj", "<i4"), ("grid", "<i4"), ("half", "<i4"), ("alpha", "<i4"),
                       ("src", "<i4"), ("dst", "<i4"), ("t", "<f8"), ("omega", "<f8")])


class AqtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libaqt.so; raise if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, D, I, I64, U64, SZ = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_int64, C.c_uint64, C.c_size_t
        sig = {
            "aqt_create": (I, [C.POINTER(P), I]),
            "aqt_destroy": (None, [P]),
            "aqt_last_error": (C.c_char_p, [P]),
            "aqt_set_ising": (I, [P, I, D, D]),
            "aqt_set_schedule": (I, [P, I, D, D, D]),
            "aqt_set_bath": (I, [P, C.c_double, C.c_double, C.c_double, I]),
            "aqt_set_levels": (I, [P, I]),
            "aqt_set_grid": (I, [P, C.c_double, I]),
            "aqt_set_trajectories": (I, [P, I64, U64, I, I, I64]),
            "aqt_workspace_size": (I, [P, C.POINTER(SZ)]),
            "aqt_bind_workspace": (I, [P, P, SZ]),
            "aqt_build_tables": (I, [P, P]),
            "aqt_get_dt_bounds": (I, [P, D, C.POINTER(C.c_int32)]),
            "aqt_set_wait_limit": (I, [P, I64]),
            "aqt_run": (I, [P, P]),
            "aqt_sync": (I, [P]),
            "aqt_get_observables": (I, [P, D, D]),
            "aqt_get_observable_sums": (I, [P, D, D]),
            "aqt_observables_from_sums": (I, [I, I64, D, D, D, D]),
            "aqt_get_rotation_error": (I, [P, D]),
            "aqt_get_leakage": (I, [P, D]),
            "aqt_get_jumps": (I, [P, C.POINTER(aqt_jump), I64, C.POINTER(I64), C.POINTER(I64)]),
            "aqt_get_final_state": (I, [P, I, D]),
            "aqt_debug_table": (I, [P, I, I, D]),
            "aqt_run_static_scratch": (I, [P, P, P, P, P, I64, P, P]),
            "aqt_batch_create": (I, [C.POINTER(P), C.POINTER(P), I]),
            "aqt_batch_destroy": (None, [P]),
            "aqt_batch_last_error": (C.c_char_p, [P]),
            "aqt_batch_workspace_size": (I, [P, C.POINTER(SZ)]),
            "aqt_batch_bind_workspace": (I, [P, P, SZ]),
            "aqt_batch_tune": (I, [P, P]),
            "aqt_batch_run": (I, [P, P]),
            "aqt_batch_sync": (I, [P, C.POINTER(C.c_int32)]),
            "aqt_batch_get_shape": (I, [P, I, C.POINTER(C.c_int32)]),
            "aqt_grad_n_params": (I, [P, C.POINTER(I)]),
            "aqt_grad_workspace_size": (I, [P, I, I64, C.POINTER(SZ)]),
            "aqt_grad_bind_workspace": (I, [P, I, I64, P, SZ]),
            "aqt_grad_forward": (I, [P, P]),
            "aqt_grad_backward": (I, [P, C.c_double, P]),
            "aqt_grad_get": (I, [P, D, I, D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _check(ctx, st):
    if st != AQT_OK:
        msg = lib().aqt_last_error(ctx).decode() if ctx else ""
        raise AqtError(st, msg)


# ---- same-name wrappers ----------------------------------------------------------
def aqt_create(device: int = 0):
    h = C.c_void_p()
    st = lib().aqt_create(C.byref(h), device)
    if st != AQT_OK:
        raise AqtError(st, f"aqt_create(device={device})")
    return h


def aqt_destroy(ctx):
    lib().aqt_destroy(ctx)


def aqt_last_error(ctx) -> str:
    return lib().aqt_last_error(ctx).decode()


def aqt_set_ising(ctx, n_qubits, hz, Jzz):
    hz, J = _f64(hz), _f64(Jzz).reshape(-1)
    _check(ctx, lib().aqt_set_ising(ctx, int(n_qubits), _dp(hz), _dp(J)))


def aqt_set_schedule(ctx, s, A, B):
    s, A, B = _f64(s), _f64(A), _f64(B)
    _check(ctx, lib().aqt_set_schedule(ctx, len(s), _dp(s), _dp(A), _dp(B)))


def aqt_set_bath(ctx, eta_g2, omega_c, beta, lamb_shift):
    _check(ctx, lib().aqt_set_bath(ctx, float(eta_g2), float(omega_c), float(beta), int(bool(lamb_shift))))


def aqt_set_levels(ctx, n_levels):
    _check(ctx, lib().aqt_set_levels(ctx, int(n_levels)))


def aqt_set_grid(ctx, t_f, n_grid):
    _check(ctx, lib().aqt_set_grid(ctx, float(t_f), int(n_grid)))


def aqt_set_trajectories(ctx, M, seed, precision, jump_timing, jump_capacity):
    _check(ctx, lib().aqt_set_trajectories(ctx, int(M), int(seed) & (2**64 - 1), int(precision),
                                           int(jump_timing), int(jump_capacity)))


def aqt_workspace_size(ctx) -> int:
    n = C.c_size_t()
    _check(ctx, lib().aqt_workspace_size(ctx, C.byref(n)))
    return n.value


def aqt_bind_workspace(ctx, dptr: int, nbytes: int):
    _check(ctx, lib().aqt_bind_workspace(ctx, C.c_void_p(dptr), nbytes))


def aqt_build_tables(ctx, stream: int = 0) -> int:
    """Returns AQT_OK, or the warning AQT_WDT (tables built and usable); raises on errors."""
    st = lib().aqt_build_tables(ctx, C.c_void_p(stream))
    if st not in (AQT_OK, AQT_WDT):
        _check(ctx, st)
    return st


def aqt_get_dt_bounds(ctx):
    """The three terms of Eq. newcond minimised over the grid (ns) and their grid points."""
    b = np.empty(3)
    at = (C.c_int32 * 3)()
    _check(ctx, lib().aqt_get_dt_bounds(ctx, _dp(b), at))
    return b, [int(x) for x in at]


def aqt_set_wait_limit(ctx, polls: int):
    _check(ctx, lib().aqt_set_wait_limit(ctx, int(polls)))


def aqt_run(ctx, stream: int = 0):
    _check(ctx, lib().aqt_run(ctx, C.c_void_p(stream)))


def aqt_sync(ctx) -> int:
    """Returns the status (AQT_OK or AQT_EOVERFLOW); raises on other errors."""
    st = lib().aqt_sync(ctx)
    if st not in (AQT_OK, AQT_EOVERFLOW):
        _check(ctx, st)
    return st


def aqt_get_observables(ctx, n_grid: int):
    mean, se = np.empty(n_grid), np.empty(n_grid)
    _check(ctx, lib().aqt_get_observables(ctx, _dp(mean), _dp(se)))
    return mean, se


def aqt_get_observable_sums(ctx, n_grid: int):
    s1, s2 = np.empty(n_grid), np.empty(n_grid)
    _check(ctx, lib().aqt_get_observable_sums(ctx, _dp(s1), _dp(s2)))
    return s1, s2


def aqt_observables_from_sums(M: int, sum_x, sum_x2):
    s1, s2 = _f64(sum_x), _f64(sum_x2)
    mean, se = np.empty(len(s1)), np.empty(len(s1))
    st = lib().aqt_observables_from_sums(len(s1), int(M), _dp(s1), _dp(s2), _dp(mean), _dp(se))
    if st != AQT_OK:
        raise AqtError(st, "aqt_observables_from_sums")
    return mean, se


def aqt_get_leakage(ctx, n_grid: int):
    out = np.empty(n_grid)
    _check(ctx, lib().aqt_get_leakage(ctx, _dp(out)))
    return out


def aqt_get_rotation_error(ctx) -> float:
    v = C.c_double()
    _check(ctx, lib().aqt_get_rotation_error(ctx, C.byref(v)))
    return v.value


def aqt_get_jumps(ctx, cap: int):
    buf = (aqt_jump * max(cap, 1))()
    n_out, n_drop = C.c_int64(), C.c_int64()
    _check(ctx, lib().aqt_get_jumps(ctx, buf, int(cap), C.byref(n_out), C.byref(n_drop)))
    arr = np.frombuffer(bytes(buf), dtype=JUMP_DTYPE)[: n_out.value].copy()
    return arr, n_drop.value


def aqt_get_final_state(ctx, basis: int, M: int, N: int):
    """N: the levels carried (basis 0) or 2^n (basis 1)."""
    out = np.empty((M, N, 2))
    _check(ctx, lib().aqt_get_final_state(ctx, int(basis), _dp(out)))
    return out[..., 0] + 1j * out[..., 1]


def aqt_debug_table(ctx, which: int, grid: int, shape):
    out = np.empty(int(np.prod(shape)))
    _check(ctx, lib().aqt_debug_table(ctx, int(which), int(grid), _dp(out)))
    return out.reshape(shape)


def aqt_run_static_scratch(ctx, stream: int, obs_sums: int, final_states: int, jumps: int, jump_capacity: int,
                           jump_count: int, status: int):
    """Device pointers (ints) for the outputs; scratch comes from the library's
    static array (see include/aqt.h)."""
    _check(ctx, lib().aqt_run_static_scratch(ctx, C.c_void_p(stream), C.c_void_p(obs_sums),
                                             C.c_void_p(final_states), C.c_void_p(jumps), int(jump_capacity),
                                             C.c_void_p(jump_count), C.c_void_p(status)))


def _bcheck(b, st):
    if st != AQT_OK:
        msg = lib().aqt_batch_last_error(b).decode() if b else ""
        raise AqtError(st, msg)


def aqt_batch_create(ctxs):
    arr = (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    h = C.c_void_p()
    st = lib().aqt_batch_create(C.byref(h), arr, len(ctxs))
    if st != AQT_OK:
        raise AqtError(st, "aqt_batch_create")
    return h


def aqt_batch_destroy(b):
    lib().aqt_batch_destroy(b)


def aqt_batch_last_error(b) -> str:
    return lib().aqt_batch_last_error(b).decode()


def aqt_batch_workspace_size(b) -> int:
    n = C.c_size_t()
    _bcheck(b, lib().aqt_batch_workspace_size(b, C.byref(n)))
    return n.value


def aqt_batch_bind_workspace(b, dptr: int, nbytes: int):
    _bcheck(b, lib().aqt_batch_bind_workspace(b, C.c_void_p(dptr), nbytes))


def aqt_batch_tune(b, stream: int = 0):
    _bcheck(b, lib().aqt_batch_tune(b, C.c_void_p(stream)))


def aqt_batch_run(b, stream: int = 0):
    _bcheck(b, lib().aqt_batch_run(b, C.c_void_p(stream)))


def aqt_batch_sync(b, n_members: int):
    """Returns (status, per-member statuses); raises on errors other than AQT_EOVERFLOW."""
    ms = (C.c_int32 * n_members)()
    st = lib().aqt_batch_sync(b, ms)
    if st not in (AQT_OK, AQT_EOVERFLOW):
        _bcheck(b, st)
    return st, [int(x) for x in ms]


def aqt_batch_get_shape(b, member: int):
    out = (C.c_int32 * 4)()
    _bcheck(b, lib().aqt_batch_get_shape(b, int(member), out))
    return tuple(int(x) for x in out)


def aqt_grad_n_params(ctx) -> int:
    n = C.c_int()
    _check(ctx, lib().aqt_grad_n_params(ctx, C.byref(n)))
    return n.value


def aqt_grad_workspace_size(ctx, checkpoint_every: int, jump_capacity: int) -> int:
    n = C.c_size_t()
    _check(ctx, lib().aqt_grad_workspace_size(ctx, int(checkpoint_every), int(jump_capacity), C.byref(n)))
    return n.value


def aqt_grad_bind_workspace(ctx, checkpoint_every: int, jump_capacity: int, dptr: int, nbytes: int):
    _check(ctx, lib().aqt_grad_bind_workspace(ctx, int(checkpoint_every), int(jump_capacity), C.c_void_p(dptr),
                                              nbytes))


def aqt_grad_forward(ctx, stream: int = 0):
    _check(ctx, lib().aqt_grad_forward(ctx, C.c_void_p(stream)))


def aqt_grad_backward(ctx, baseline: float = float("nan"), stream: int = 0):
    _check(ctx, lib().aqt_grad_backward(ctx, float(baseline), C.c_void_p(stream)))


def aqt_grad_get(ctx, n_params: int):
    g = np.empty(n_params)
    v = C.c_double()
    _check(ctx, lib().aqt_grad_get(ctx, _dp(g), int(n_params), C.byref(v)))
    return g, v.value


# ---- convenience ------------------------------------------------------------------
class Session:
    """One context configured from an instance (see ``workloads.Instance``),
    with its workspace held as a torch uint8 tensor on the context's device."""

    def __init__(self, inst, precision=AQT_PREC_FP64, jump_capacity=None, device=0, M=None, seed=None,
                 timing=AQT_JUMP_REFINED):
        self.inst = inst
        self.device = device
        self.M = int(inst.M if M is None else M)
        self.D = 1 << inst.n_qubits
        nl = int(getattr(inst, "n_levels", 0) or 0)
        self.N = nl if 0 < nl < self.D else self.D
        self.K = inst.n_grid
        self.ctx = aqt_create(device)
        self.jcap = int(jump_capacity if jump_capacity is not None else max(1024, 64 * self.M))
        self.configure(inst, precision, seed, timing)
        self.ws = None

    def configure(self, inst, precision, seed=None, timing=AQT_JUMP_REFINED):
        c = self.ctx
        aqt_set_ising(c, inst.n_qubits, inst.hz, inst.J)
        aqt_set_schedule(c, inst.sched_s, inst.sched_A, inst.sched_B)
        aqt_set_bath(c, inst.eta_g2, inst.omega_c, inst.beta, inst.lamb_shift)
        aqt_set_levels(c, int(getattr(inst, "n_levels", 0) or 0))
        aqt_set_grid(c, inst.t_f, inst.n_grid)
        aqt_set_trajectories(c, self.M, inst.seed if seed is None else seed, precision, timing, self.jcap)

    def allocate(self):
        import torch
        nbytes = aqt_workspace_size(self.ctx)
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{self.device}")
        aqt_bind_workspace(self.ctx, self.ws.data_ptr(), self.ws.numel())

    @staticmethod
    def stream() -> int:
        import torch
        return torch.cuda.current_stream().cuda_stream

    def build(self):
        self.allocate()
        return aqt_build_tables(self.ctx, self.stream())

    def run(self):
        aqt_run(self.ctx, self.stream())
        return aqt_sync(self.ctx)

    def observables(self):
        return aqt_get_observables(self.ctx, self.K)

    def jumps(self):
        return aqt_get_jumps(self.ctx, self.jcap)

    def final_state(self, basis=1):
        return aqt_get_final_state(self.ctx, basis, self.M, self.D if basis == 1 else self.N)

    def grad_allocate(self, checkpoint_every=64, jump_capacity=None):
        """Bind a gradient workspace (torch uint8 tensor on the context's device)."""
        import torch
        jc = int(jump_capacity if jump_capacity is not None else max(1024, 4 * self.M))
        nbytes = aqt_grad_workspace_size(self.ctx, checkpoint_every, jc)
        if getattr(self, "gws", None) is None or self.gws.numel() < nbytes:
            self.gws = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{self.device}")
        aqt_grad_bind_workspace(self.ctx, checkpoint_every, jc, self.gws.data_ptr(), self.gws.numel())

    def gradient(self, baseline=float("nan"), checkpoint_every=64, jump_capacity=None):
        """Forward run with checkpoints and the adjoint sweep; returns
        (d<P>/dtheta, <P>) for P the ground-manifold population at s = 1."""
        self.grad_allocate(checkpoint_every, jump_capacity)
        aqt_grad_forward(self.ctx, self.stream())
        aqt_grad_backward(self.ctx, baseline, self.stream())
        return aqt_grad_get(self.ctx, aqt_grad_n_params(self.ctx))

    def close(self):
        if self.ctx:
            aqt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
