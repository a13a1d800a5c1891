"""splitmix64 counter-based generator (Steele, Lea & Flood, OOPSLA 2014; constants as in
Vigna's public reference splitmix64.c), used for the power-iteration start vector so that
the oracle and the CUDA library start from the same vector without sharing code.

Output i of the stream seeded with s is mix(s + (i + 1) * 0x9E3779B97F4A7C15 mod 2^64),
mix(z) = z1 ^ (z1 >> 31) where z1 = (z0 ^ (z0 >> 27)) * 0x94D049BB133111EB and
z0 = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 (all mod 2^64).
uniform_pm1(s, n)[i] = 2 * ((output_i >> 11) * 2^-53) - 1, in [-1, 1).

TEST INFRASTRUCTURE: only tests, smoke() and the bench CPU baseline use this module.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of the splitmix64 stream started at `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n float64 values in [-1, 1) from splitmix64."""
    z = splitmix64(seed, n)
    return 2.0 * ((z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)) - 1.0
