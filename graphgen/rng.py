"""Counter-based random numbers for the synthetic inputs.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) evaluated on a counter: draw ``i`` of stream
``(seed, stream)`` is ``mix(seed_key + (i + 1) * GOLDEN)``, with ``seed_key``
itself a SplitMix64 hash of ``(seed, stream)``. Being counter-based, any slice
of a stream can be produced independently and the values do not depend on the
numpy version or the machine, so the CPU and GPU machines build bit-identical
graphs from the same seed.

This module holds no part of the resistance-distance method; it only makes
inputs.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        a = _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64) + _GOLDEN)
        b = _mix(a ^ np.uint64(stream & 0xFFFFFFFFFFFFFFFF))
    return b[0]


def bits(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` raw 64-bit draws ``offset .. offset+count-1`` of a stream."""
    key = _key(seed, stream)
    ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + ctr * _GOLDEN)


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles uniform on [0, 1) with 53 random bits."""
    return (bits(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def integers(seed: int, stream: int, count: int, high: int, offset: int = 0) -> np.ndarray:
    """Integers uniform on [0, high) (multiply-shift; bias below 2**-20 for high < 2**32)."""
    if high <= 0:
        raise ValueError("high must be positive")
    u = uniform(seed, stream, count, offset)
    return np.minimum((u * high).astype(np.int64), high - 1)


def normal(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform of two uniform streams."""
    u1 = uniform(seed, stream, count, offset)
    u2 = uniform(seed, stream + 0x5BD1E995, count, offset)
    u1 = 1.0 - u1  # (0, 1]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
