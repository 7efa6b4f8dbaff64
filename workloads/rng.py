"""Counter-based pseudo-random numbers for the synthetic workloads.

Every random draw of the workloads is a pure function of (seed, stream tag,
counter), so any element can be regenerated on its own, in any order, and a
vectorised numpy evaluation gives the same numbers as a scalar loop would.

The bit generator is the SplitMix64 output function (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014; constants as
published by Vigna for ``splitmix64.c``) applied to ``key + (counter + 1) *
0x9E3779B97F4A7C15``.  A uniform double in [0, 1) takes the top 53 bits.

Nothing here computes any part of the sparse-matrix method: this module only
makes inputs.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30 = np.uint64(30)
_S27 = np.uint64(27)
_S31 = np.uint64(31)
_S11 = np.uint64(11)
_INV53 = 1.0 / float(1 << 53)


def mix64(z):
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _S30)) * _M1
        z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def stream_key(seed: int, *tags: int) -> np.uint64:
    """Key of one independent stream, derived from a base seed and integer tags."""
    k = mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    for t in tags:
        with np.errstate(over="ignore"):
            k = mix64(k ^ mix64(np.uint64(t & 0xFFFFFFFFFFFFFFFF) + _GOLDEN))
    return np.uint64(k)


def bits(key, ctr):
    """64 random bits for each counter value in ``ctr`` (int array)."""
    c = np.asarray(ctr).astype(np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (c + np.uint64(1)) * _GOLDEN
    return mix64(z)


def uniform01(key, ctr):
    """Uniform doubles in [0, 1), 53-bit resolution."""
    return (bits(key, ctr) >> _S11).astype(np.float64) * _INV53


def uniform(key, ctr, lo: float, hi: float):
    """Uniform doubles in [lo, hi)."""
    return lo + (hi - lo) * uniform01(key, ctr)


def randint(key, ctr, lo: int, hi: int):
    """Uniform integers in the closed range [lo, hi] (hi - lo < 2**52)."""
    n = hi - lo + 1
    return lo + np.floor(uniform01(key, ctr) * n).astype(np.int64)


def normal(key, ctr):
    """Standard normal doubles by the Box-Muller transform of two uniforms."""
    c = np.asarray(ctr).astype(np.int64)
    u1 = 1.0 - uniform01(key, 2 * c)  # (0, 1]
    u2 = uniform01(key, 2 * c + 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
