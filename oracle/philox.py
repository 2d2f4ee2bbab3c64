"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel
random numbers: as easy as 1, 2, 3"), written out from its published definition.

One call maps a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1) to four
32-bit words.  Each of the 10 rounds multiplies c0 and c2 by the two round
multipliers, exchanges and xors the halves with the key, then bumps the key by
the two Weyl constants.  Vectorised over numpy arrays of counters.
"""
from __future__ import annotations

import numpy as np

ROUND_MUL_0 = 0xD2511F53
ROUND_MUL_1 = 0xCD9E8D57
WEYL_0 = 0x9E3779B9
WEYL_1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF


def philox4x32(c0, c1, c2, c3, k0, k1, rounds: int = 10):
    """Return the four output words (uint32 arrays) for the given counters and key."""
    c0, c1, c2, c3 = np.broadcast_arrays(*(np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3)))
    c0, c1, c2, c3 = (x.copy() for x in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & MASK32)
    k1 = np.uint64(int(k1) & MASK32)
    m0 = np.uint64(ROUND_MUL_0)
    m1 = np.uint64(ROUND_MUL_1)
    mask = np.uint64(MASK32)
    s32 = np.uint64(32)
    for _ in range(rounds):
        p0 = c0 * m0            # 64-bit product of two 32-bit values: exact in uint64
        p1 = c2 * m1
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(WEYL_0)) & mask
        k1 = (k1 + np.uint64(WEYL_1)) & mask
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def key_of(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & MASK32, seed >> 32


def uniform23(word) -> np.ndarray:
    """Map a 32-bit word to a uniform in (0, 1): ((w >> 9) + 0.5) * 2**-23.

    The result is exactly representable in float32, so the CUDA path (which uses
    the same map) and this oracle start every derived quantity from identical
    uniforms."""
    w = np.asarray(word, dtype=np.uint64)
    return ((w >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23
