"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as
1, 2, 3", SC'11), written from its published definition with numpy uint64 lanes.

One call maps a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1) to four
uint32 words.  A round multiplies c0 and c2 by the two Philox multipliers, keeps
the high and low halves, and permutes/XORs them with c1, c3 and the key; the key is
bumped by the two Weyl constants between rounds (10 rounds, 9 bumps).

Counter convention of the method (both sides use it): c0 = draw index, c1 = entity
index (cut node, column, ...), c2 = slice, c3 = purpose tag; key = the 64-bit seed.
"""
from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)

# purpose tags (counter word c3)
TAG_PASS1 = 1
TAG_PASS2 = 2
TAG_ALSINIT = 3


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10. Arguments broadcast; returns four uint32 arrays."""
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(
        *[np.asarray(x, dtype=np.uint64) & MASK32 for x in (c0, c1, c2, c3, k0, k1)])
    c0, c1, c2, c3, k0, k1 = (x.copy() for x in (c0, c1, c2, c3, k0, k1))
    for r in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r < 9:
            k0 = (k0 + _W0) & MASK32
            k1 = (k1 + _W1) & MASK32
    return (c0.astype(np.uint32), c1.astype(np.uint32), c2.astype(np.uint32), c3.astype(np.uint32))


def seed_key(seed: int):
    """Split a 64-bit seed into the Philox key words (low, high)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def draw(seed: int, t, entity, slice_id, tag):
    """Philox output words for counter (t, entity, slice, tag) under ``seed``."""
    k0, k1 = seed_key(seed)
    return philox4x32_10(t, entity, slice_id, tag, k0, k1)


def uniform_index(word, size: int):
    """Map a uint32 word to an index in [0, size): floor(word * size / 2^32)."""
    return ((np.asarray(word, dtype=np.uint64) * np.uint64(size)) >> np.uint64(32)).astype(np.int64)
