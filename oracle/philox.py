"""Philox4x32-10 counter-based random numbers, from the published definition
(Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).

The paper draws the Rademacher diagonal R and the column subsample P of Definition 1
(Sec. 3.2) at random but names no generator.  Reading used here and by the CUDA path:
a 4x32 Philox with 10 rounds, key = (seed mod 2^32, seed div 2^32), counter =
(index mod 2^32, index div 2^32, stream, 0).

Test infrastructure (see the package docstring).
"""
import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10_block(c0, c1, c2, c3, k0, k1):
    """The generator's block function on a full counter (c0, c1, c2, c3) and key (k0, k1),
    all 32-bit words (uint64 arrays or scalars); returns the four output words.

    One round: (c0, c1, c2, c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
    hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)); the key is bumped by the Weyl constants
    (W0, W1) before every round after the first.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def philox4x32_10(index, stream, seed):
    """Return the four 32-bit output words (as uint64 arrays) for counters
    (index_lo, index_hi, stream, 0) under key (seed_lo, seed_hi)."""
    index = np.asarray(index, dtype=np.uint64)
    c0 = index & _MASK
    c1 = index >> np.uint64(32)
    c2 = np.full_like(c0, np.uint64(stream) & _MASK)
    c3 = np.zeros_like(c0)
    return philox4x32_10_block(c0, c1, c2, c3, int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)
