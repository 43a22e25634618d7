"""SplitMix64 counter-based generator (Steele, Lea & Flood, OOPSLA 2014).

The paper leaves the Lanczos start vector unspecified (Section 3.4).  Both the
oracle and the GPU library draw it from this generator so that their
eigenvalue estimates start from the same vector: element i is the (i+1)-th
output of SplitMix64 seeded with ``seed``, mapped to [-1, 1) exactly as
2 * (z >> 11) * 2^-53 - 1.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first n outputs of SplitMix64 started from state ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + _GOLDEN * np.arange(1, n + 1, dtype=np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    z = splitmix64(seed, n)
    return 2.0 * ((z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53) - 1.0
