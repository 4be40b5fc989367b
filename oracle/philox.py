"""Oracle (test infrastructure only): Philox4x32-10 counter-based generator.

Written from its published definition (Salmon, Moraes, Dror & Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC 2011): a 4x32-bit counter and 2x32-bit key,
ten rounds; each round multiplies counter words 0 and 2 by fixed 32-bit constants,
swaps and xors the high halves with the other words and the round key, and the key
is bumped by two Weyl constants between rounds.

The GPU path carries its own implementation of the same definition; neither side
imports the other. Arrays are numpy uint64 holding 32-bit values.
"""
import numpy as np

MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words for counters (c0..c3) under key (k0, k1)."""
    c0, c1, c2, c3, k0, k1 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3, k0, k1))
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & MASK
            k1 = (k1 + _W1) & MASK
        p0 = _M0 * c0          # < 2^64: exact in uint64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & MASK
        hi1, lo1 = p1 >> _S32, p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform_open(word):
    """Map a 32-bit word to (0, 1): (2 * (w >> 9) + 1) * 2^-24, exactly representable in FP32 and FP64."""
    w = np.asarray(word, dtype=np.uint64)
    return (2.0 * (w >> np.uint64(9)).astype(np.float64) + 1.0) * 2.0 ** -24
