"""Ohmic bath rates and Lamb shift.

Test infrastructure only (see the package docstring).

Sec. V: gamma(omega) = 2 pi eta g^2 omega exp(-|omega|/omega_c) / (1 - exp(-beta omega)),
which obeys the KMS condition gamma(-omega) = exp(-beta omega) gamma(omega)
(Sec. II, Eq. KMS). At omega = 0 the limit 2 pi eta g^2 / beta is used.

The Lamb shift H_LS = sum_{alpha,omega} S(omega) L^dag L (Sec. II; App. E) is
named but not written out in the paper. Reading: S is the principal-value
transform of the same spectral density, S(omega) = (1/2pi) P int gamma(x) / (omega - x) dx
(the imaginary part of the one-sided bath correlation integral). Here it is
evaluated by QUADPACK's Cauchy-weight rule on a node table and interpolated by
a cubic spline.
"""
from __future__ import annotations

import functools
import math
import multiprocessing
import os

import numpy as np
from scipy import integrate, interpolate


def gamma(omega, eta_g2: float, omega_c: float, beta: float):
    """Ohmic rate gamma(omega) in 1/ns for omega in rad/ns (Sec. V)."""
    w = np.asarray(omega, dtype=float)
    out = np.empty_like(w)
    zero = w == 0.0
    wz = np.where(zero, 1.0, w)
    # omega / (1 - exp(-beta omega)) written as omega / (-expm1(-beta omega)).
    with np.errstate(over="ignore"):
        out = 2.0 * math.pi * eta_g2 * wz * np.exp(-np.abs(wz) / omega_c) / (-np.expm1(-beta * wz))
    out = np.where(zero, 2.0 * math.pi * eta_g2 / beta, out)
    return out if out.ndim else float(out)


def _support(omega_c: float, beta: float) -> float:
    # gamma decays like exp(-|x|/omega_c) for x > 0 and faster for x < 0;
    # beyond 60 omega_c the neglected tail is below 1e-22 of the peak.
    return 60.0 * omega_c


def lamb_shift_direct(omega: float, eta_g2: float, omega_c: float, beta: float) -> float:
    """S(omega) by one principal-value quadrature (slow; used for tables and pins).

    The pole is removed by subtraction: over [-L, L],
      P int g(x)/(omega - x) dx = int (g(x) - g(omega))/(omega - x) dx
                                  + g(omega) ln((omega + L)/(L - omega)),
    and the bounded remainder goes to QUADPACK with breakpoints at the pole and
    at the kink of gamma at 0.
    """
    L = _support(omega_c, beta)
    g0 = gamma(omega, eta_g2, omega_c, beta)

    def f(x):
        if x == omega:   # removable point of the subtracted integrand (measure zero)
            return 0.0
        return (gamma(x, eta_g2, omega_c, beta) - g0) / (omega - x)

    pts = sorted(set(p for p in (omega, 0.0, -omega_c, omega_c) if -L < p < L))
    edges = [-L] + pts + [L]
    total = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        v, _ = integrate.quad(f, lo, hi, limit=200, epsabs=1e-16, epsrel=1e-13)
        total += v
    total += g0 * math.log((omega + L) / (L - omega))
    return total / (2.0 * math.pi)


def _lamb_nodes(wmax: float) -> np.ndarray:
    # Disjoint node ranges (no near-duplicate nodes): fine near 0, where S has
    # logarithmic curvature from the kink of gamma, medium up to |omega| = 10
    # (the thermal factor varies on the scale 1/beta), coarse beyond (omega_c).
    inner = np.linspace(0.0, 0.05, 201)
    mid = np.linspace(0.05, 10.0, 500)[1:]
    far = np.linspace(10.0, max(wmax, 10.5), max(2, int(np.ceil((wmax - 10.0) / 0.5)) + 1))[1:]
    pos = np.concatenate([inner, mid, far])
    return np.concatenate([-pos[:0:-1], pos])


def _lamb_node_values(args):
    nodes, eta_g2, omega_c, beta = args
    return [lamb_shift_direct(float(w), eta_g2, omega_c, beta) for w in nodes]


@functools.lru_cache(maxsize=16)
def _lamb_spline(eta_g2: float, omega_c: float, beta: float, wmax: float):
    nodes = _lamb_nodes(wmax)
    # A spawn pool only from the main process (a worker never starts another).
    workers = max(1, min(16, os.cpu_count() or 1))
    if multiprocessing.current_process().name != "MainProcess":
        workers = 1
    chunks = [(c, eta_g2, omega_c, beta) for c in np.array_split(nodes, 4 * workers)]
    if workers > 1:
        ctx = multiprocessing.get_context("spawn")
        with ctx.Pool(workers) as pool:
            vals = np.concatenate([np.array(v) for v in pool.map(_lamb_node_values, chunks)])
    else:
        vals = np.concatenate([np.array(_lamb_node_values(c)) for c in chunks])
    return interpolate.CubicSpline(nodes, vals)


def lamb_shift(omega, eta_g2: float, omega_c: float, beta: float, wmax: float = 400.0):
    """S(omega) in rad/ns from the interpolated node table (|omega| <= wmax)."""
    w = np.asarray(omega, dtype=float)
    if np.any(np.abs(w) > wmax):
        raise ValueError("Bohr frequency outside the Lamb-shift table")
    wmax = float(np.ceil(wmax / 50.0) * 50.0)
    return _lamb_spline(float(eta_g2), float(omega_c), float(beta), wmax)(w)
