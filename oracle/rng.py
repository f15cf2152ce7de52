"""SplitMix64 counter generator and Rademacher probes (oracle side).

Test infrastructure only.  SplitMix64 (Steele, Lea & Flood, OOPSLA 2014):
state advances by GAMMA = 0x9E3779B97F4A7C15 and each output is the state
passed through the variant-13 finaliser.  Output i of the stream seeded with
``s`` is therefore mix(s + (i + 1) * GAMMA), so any draw can be computed from
its index alone.

Seeded SLQ probes: entry (v, i) of the probe block for an operator of size N
is output v * N + i of the stream; it is +1 when the top bit is 0, else -1.
"""
from __future__ import annotations

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def output(seed: int, i: int) -> int:
    return mix((seed + (i + 1) * GAMMA) & MASK)


def rademacher_probes(seed: int, nprobes: int, N: int):
    """Probe block (nprobes, N) as a numpy float64 array."""
    import numpy as np
    idx = np.arange(1, nprobes * N + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK) + idx * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return np.where((z >> np.uint64(63)) == 0, 1.0, -1.0).reshape(nprobes, N)
