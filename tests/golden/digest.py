"""Order-independent digest of a set of 64-bit state vectors (test utility).

digest(S) = (|S|, sum of f(x) mod 2^64, xor of f(x)) with f the SplitMix64
output finaliser (a bijection), so two sets with equal digests are equal with
overwhelming probability.  Used to compare the CUDA path's BFS levels with
stored oracle levels at sizes too large to keep the oracle's states.
"""
import numpy as np


def _f(x):
    z = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def digest(states):
    s = np.asarray(states).astype(np.uint64, copy=False)
    if s.size == 0:
        return [0, 0, 0]
    f = _f(s)
    with np.errstate(over="ignore"):
        total = int(np.add.reduce(f, dtype=np.uint64))
    return [int(s.size), total, int(np.bitwise_xor.reduce(f))]
