"""Counter-based uniform noise.

splitmix64 is the 64-bit finaliser published by Steele, Lea & Flood
("Fast splittable pseudorandom number generators", OOPSLA 2014), in the form
popularised by S. Vigna.  A value depends only on (seed, field_id, cell index),
so any subset of cells can be regenerated independently and both sides of a
comparison see identical inputs.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied element-wise to uint64 counters."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, field_id: int, count: int, index=None) -> np.ndarray:
    """xi in [-1, 1) from the top 53 bits of splitmix64(seed ^ field_id*2^40 ^ index).

    ``index`` defaults to 0..count-1 (linear cell index (k*nth + j)*nr + i).
    """
    if index is None:
        index = np.arange(count, dtype=np.uint64)
    else:
        index = np.asarray(index, dtype=np.uint64)
    key = np.uint64(seed) ^ (np.uint64(field_id) << np.uint64(40))
    bits = splitmix64(index ^ key) >> np.uint64(11)
    return bits.astype(np.float64) * (2.0 ** -52) - 1.0
