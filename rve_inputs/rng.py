"""SplitMix64 as a counter-based generator (vectorised with numpy uint64).

Value i of stream `seed` is mix(seed + (i + 1) * GAMMA), which is exactly the
i-th output of the sequential SplitMix64 generator started from state `seed`.
"""

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count, offset=0):
    """Return `count` raw 64-bit outputs of SplitMix64 seeded with `seed`,
    starting at output index `offset`."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, count, offset=0):
    """Uniform doubles in the open interval (0, 1): ((z >> 11) + 0.5) * 2^-53."""
    z = splitmix64(seed, count, offset)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def standard_normal(seed, count, offset=0):
    """Standard normal doubles by the Box-Muller transform of consecutive pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m, offset)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * np.pi * u2
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    return out[:count]
