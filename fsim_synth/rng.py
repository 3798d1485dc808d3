"""SplitMix64 counter-based generator (Steele, Lea & Flood, OOPSLA 2014).

Every synthetic input in this repository (geometries, exponents, raw
contraction coefficients, network initial weights) is drawn from this stream,
so the CUDA path and the CPU oracle see bit-identical inputs.  Nothing in this
module performs any step of the Hartree-Fock method.
"""
from __future__ import annotations

import math

_MASK = (1 << 64) - 1


class SplitMix64:
    """64-bit SplitMix generator with a few convenience draws."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 53 bits."""
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def uniform_open_low(self, lo: float, hi: float) -> float:
        """Uniform double in (lo, hi]."""
        u = ((self.next_u64() >> 11) + 1) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in the closed range [lo, hi]."""
        n = hi - lo + 1
        return lo + int(self.uniform() * n) % n

    def normal(self) -> float:
        """Standard normal by Box-Muller (one value per two uniforms)."""
        u1 = self.uniform_open_low(0.0, 1.0)
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def choice(self, weights) -> int:
        """Index drawn with the given (unnormalised) probabilities."""
        total = float(sum(weights))
        x = self.uniform() * total
        acc = 0.0
        for i, w in enumerate(weights):
            acc += w
            if x < acc:
                return i
        return len(weights) - 1

    def shuffle(self, seq: list) -> list:
        """Fisher-Yates shuffle in place; returns the list."""
        for i in range(len(seq) - 1, 0, -1):
            j = self.randint(0, i)
            seq[i], seq[j] = seq[j], seq[i]
        return seq
