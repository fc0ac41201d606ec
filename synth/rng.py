"""Counter-based pseudo-random numbers shared by the oracle, the tests and the bench.

Every draw is a pure function of (seed, stream name, counter), so the same inputs are
produced on any machine (x86 build host, Arm GPU host) and with any numpy version.
The generator is SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used in counter mode: value i of a stream is the SplitMix64
output function applied to key + (i + 1) * golden_gamma.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _fnv1a64(text: str) -> int:
    h = 0xCBF29CE484222325
    for byte in text.encode("utf-8"):
        h ^= byte
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


class Stream:
    """One named stream of a seed; successive calls continue the counter."""

    def __init__(self, seed: int, name: str):
        k = np.array([(int(seed) * 0x9E3779B97F4A7C15 ^ _fnv1a64(name)) & 0xFFFFFFFFFFFFFFFF],
                     dtype=np.uint64)
        self._key = _mix(k)[0]
        self._ctr = 0

    def bits(self, n: int) -> np.ndarray:
        i = np.arange(self._ctr + 1, self._ctr + 1 + n, dtype=np.uint64)
        self._ctr += n
        with np.errstate(over="ignore"):
            return _mix(self._key + i * _GAMMA)

    def bits_at(self, idx) -> np.ndarray:
        """Values at explicit counter positions idx (0-based; does not advance the stream):
        bits_at(range(c, c + n)) equals the next n values of a stream at counter c."""
        i = np.asarray(idx, dtype=np.uint64) + np.uint64(1)
        with np.errstate(over="ignore"):
            return _mix(self._key + i * _GAMMA)

    def uniform_at(self, idx, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.bits_at(idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """n doubles in [lo, hi): the top 53 bits scaled by 2**-53."""
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def integers(self, n: int, hi: int) -> np.ndarray:
        """n integers in [0, hi) (multiply-shift on the top 32 bits; bias < 2**-32 * hi)."""
        top = (self.bits(n) >> np.uint64(32)).astype(np.uint64)
        return ((top * np.uint64(hi)) >> np.uint64(32)).astype(np.int64)

    def permutation(self, n: int) -> np.ndarray:
        """Fisher-Yates shuffle of range(n) driven by this stream."""
        p = np.arange(n, dtype=np.int64)
        r = self.uniform(max(n - 1, 0))
        for t, i in enumerate(range(n - 1, 0, -1)):
            j = int(r[t] * (i + 1))
            p[i], p[j] = p[j], p[i]
        return p

    def normal(self, n: int) -> np.ndarray:
        """Standard normal deviates by the Box-Muller transform."""
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
