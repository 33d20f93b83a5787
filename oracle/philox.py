"""Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), written from the
published round function, and the random-stream layout of one trajectory.

Test infrastructure only (see the package docstring).

Stream layout (a reading: the paper only says "draw a random number", Sec. IV):
  key     = (seed, 0x0000000171003431)
  counter = (trajectory index, event index, 0, 0)
  event 0          -> x0: first jump threshold r
  event j >= 1     -> x0: u1 (source draw), x1: u2 (target draw),
                      x2: threshold r after the j-th jump
  uniform(x)       = ((x >> 12) + 0.5) * 2**-52, strictly inside (0, 1)
Fixed-step sampler (App. B.1), one block per frozen piece q of the grid:
  counter = (trajectory index, q, 1, 0) -> x0: eps (jump test), x1: u1, x2: u2
                     (every value is a multiple of 2**-53, so exact in FP64)
"""
from __future__ import annotations

MASK64 = (1 << 64) - 1
# Round multipliers and Weyl key increments of Philox4x64 (SC'11, Table 2).
_M0 = 0xD2E7470EE14C6C93
_M1 = 0xCA5A826395121157
_W0 = 0x9E3779B97F4A7C15
_W1 = 0xBB67AE8584CAA73B
KEY_HI = 0x0000000171003431


def philox4x64(counter, key, rounds: int = 10):
    """Return the four 64-bit outputs for a 4x64-bit counter and 2x64-bit key."""
    x0, x1, x2, x3 = (int(c) & MASK64 for c in counter)
    k0, k1 = (int(k) & MASK64 for k in key)
    for _ in range(rounds):
        p0 = _M0 * x0
        p1 = _M1 * x2
        x0, x1, x2, x3 = ((p1 >> 64) ^ x1 ^ k0, p1 & MASK64,
                          (p0 >> 64) ^ x3 ^ k1, p0 & MASK64)
        k0 = (k0 + _W0) & MASK64
        k1 = (k1 + _W1) & MASK64
    return x0, x1, x2, x3


def uniform(x: int) -> float:
    """Map 64 random bits to a double strictly inside (0, 1)."""
    return ((x >> 12) + 0.5) * (2.0 ** -52)


def event_block(seed: int, traj: int, event: int):
    return philox4x64((traj, event, 0, 0), (seed, KEY_HI))


def first_threshold(seed: int, traj: int) -> float:
    return uniform(event_block(seed, traj, 0)[0])


def jump_draws(seed: int, traj: int, j: int):
    """(u1, u2, r_next) for the j-th jump (j >= 1) of a trajectory."""
    x = event_block(seed, traj, j)
    return uniform(x[0]), uniform(x[1]), uniform(x[2])


def fixed_step_draws(seed: int, traj: int, piece: int):
    """(eps, u1, u2) of the fixed-step sampler for frozen piece ``piece``."""
    x = philox4x64((traj, piece, 1, 0), (seed, KEY_HI))
    return uniform(x[0]), uniform(x[1]), uniform(x[2])

