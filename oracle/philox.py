"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as
easy as 1, 2, 3", SC'11, Sec. 3.3 and Table 2), written from its published
definition.  Oracle-side implementation; the CUDA library has its own.

One round maps the counter (c0, c1, c2, c3) with round key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
and the key is bumped by the Weyl constants between rounds.  Ten rounds.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, key):
    """Vectorised Philox4x32-10.  ``c*`` are integer arrays (or scalars)
    holding 32-bit counter words; ``key`` is the 64-bit seed, split into
    k0 = low word, k1 = high word.  Returns four uint64 arrays holding the
    32-bit output words."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK
    c1 = np.asarray(c1, dtype=np.uint64) & MASK
    c2 = np.asarray(c2, dtype=np.uint64) & MASK
    c3 = np.asarray(c3, dtype=np.uint64) & MASK
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(key) & MASK)
    k1 = np.uint64((int(key) >> 32) & MASK)
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    msk = np.uint64(MASK)
    s32 = np.uint64(32)
    for rnd in range(10):
        if rnd:
            k0 = np.uint64((int(k0) + W0) & MASK)
            k1 = np.uint64((int(k1) + W1) & MASK)
        p0 = m0 * c0          # < 2^64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & msk
        hi1, lo1 = p1 >> s32, p1 & msk
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def philox_scalar(c0, c1, c2, c3, key):
    """Pure-Python Philox4x32-10 for one counter (used to cross-check the
    vectorised form on a few counters)."""
    k0, k1 = key & MASK, (key >> 32) & MASK
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & MASK, p1 & MASK, \
            ((p0 >> 32) ^ c3 ^ k1) & MASK, p0 & MASK
    return c0, c1, c2, c3
