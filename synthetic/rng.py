"""SplitMix64: the counter-based generator every synthetic input is drawn from.

Definition (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): the state advances by the golden-gamma 0x9E3779B97F4A7C15 and each
output is the state passed through the variant-13 finaliser.  Every object of a
scene draws from its own substream, seeded from the config seed and the object's
index, so adding an object never perturbs the others.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


class SplitMix64:
    """Sequential SplitMix64 stream."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _MASK
        return _mix(self.state)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def normal(self) -> float:
        """Standard normal by Box-Muller on two uniforms."""
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        return float(np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2))

    def substream(self, index: int) -> "SplitMix64":
        """Independent stream for object `index` (seed mixed with the index)."""
        return SplitMix64(_mix((self.state ^ _mix(index + 1)) & _MASK))


def uniform_array(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the vectorised counter form: output k is
    mix(seed + (k + 1) * gamma), identical to n sequential next_u64 calls."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + k * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def normal_array(seed: int, n: int) -> np.ndarray:
    """n standard normals (Box-Muller over 2n counter-form uniforms)."""
    u = uniform_array(seed, 2 * n)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
