"""Philox4x32-10 (test infrastructure; see the package header).

Written from the generator's published definition (Salmon, Moraes, Dror,
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 128-bit
counter (four 32-bit words) and a 64-bit key (two words); each of the 10
rounds multiplies words 0 and 2 by fixed odd constants, takes the 64-bit
products apart into high and low halves, and recombines them with the other
two words and the round key; the key is advanced by two Weyl constants
between rounds.

The Weyl increments are the 32-bit fractional parts of the golden ratio and
of sqrt(3) (checked against those closed forms in the tests). The two
multipliers were chosen by the generator's authors by search and have no
closed form.
"""
from __future__ import annotations

import numpy as np

MUL0 = 0xD2511F53
MUL1 = 0xCD9E8D57
WEYL0 = 0x9E3779B9   # floor(2**32 * (sqrt(5) - 1) / 2)
WEYL1 = 0xBB67AE85   # floor(2**32 * (sqrt(3) - 1))
ROUNDS = 10
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32(c0, c1, c2, c3, k0, k1, rounds: int = ROUNDS):
    """Vectorised Philox4x32-R. All arguments are broadcastable integer arrays
    (values taken mod 2**32); returns four uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    m0 = np.uint64(MUL0)
    m1 = np.uint64(MUL1)
    w0 = np.uint64(WEYL0)
    w1 = np.uint64(WEYL1)
    for r in range(rounds):
        if r:
            k0 = (k0 + w0) & _MASK
            k1 = (k1 + w1) & _MASK
        p0 = m0 * c0            # < 2**64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def edge_sign_bits(seed: int, i, j, k: int) -> np.ndarray:
    """Random signs of the projection for the unordered edges (i, j), i < j.

    For edge (i, j) and projection row r, the sign is bit (r mod 32) of word
    ((r mod 128) // 32) of Philox4x32-10 at counter (i, j, r // 128, 0) with
    key (seed mod 2**32, seed >> 32). Returns a bool array (len, k): True
    means +1/sqrt(k), False means -1/sqrt(k)."""
    i = np.asarray(i, dtype=np.uint64).ravel()
    j = np.asarray(j, dtype=np.uint64).ravel()
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    out = np.empty((i.size, k), dtype=bool)
    for rb in range((k + 127) // 128):
        words = np.stack(philox4x32(i, j, rb, 0, k0, k1), axis=1).astype("<u4")   # (N, 4)
        # bit b of word w is projection row 128 rb + 32 w + b
        bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")      # (N, 128)
        r1 = min(k, rb * 128 + 128)
        out[:, rb * 128:r1] = bits[:, :r1 - rb * 128].astype(bool)
    return out
