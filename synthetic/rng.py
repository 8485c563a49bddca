"""SplitMix64 (Steele, Lea, Flood 2014; constants as published by Vigna).

The generator is counter based: output k of stream `seed` is
mix(seed + (k + 1) * GOLDEN).  Uniforms on [-1, 1) use the top 53 bits;
normals use the Box-Muller transform on two consecutive uniforms in (0, 1].
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Stateful wrapper: successive calls continue the same stream."""

    def __init__(self, seed):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, count):
        with np.errstate(over="ignore"):
            k = np.arange(1, count + 1, dtype=np.uint64)
            z = self.state + k * _GOLDEN
            self.state = self.state + np.uint64(count) * _GOLDEN
            return _mix(z)

    def uniform01_open0(self, count):
        """Uniforms in (0, 1] with 53-bit resolution."""
        u = (self.next_u64(count) >> np.uint64(11)).astype(np.float64)
        return (u + 1.0) * (1.0 / 9007199254740992.0)

    def uniform_pm1(self, count):
        """Uniforms in [-1, 1) with 53-bit resolution."""
        u = (self.next_u64(count) >> np.uint64(11)).astype(np.float64)
        return u * (2.0 / 9007199254740992.0) - 1.0

    def standard_normal(self, count):
        m = (count + 1) // 2
        u = self.uniform01_open0(2 * m)
        u1, u2 = u[0::2], u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * m)
        z[0::2] = r * np.cos(2.0 * np.pi * u2)
        z[1::2] = r * np.sin(2.0 * np.pi * u2)
        return z[:count]


def uniform_pm1(seed, count):
    return SplitMix64(seed).uniform_pm1(count)


def standard_normal(seed, count):
    return SplitMix64(seed).standard_normal(count)
