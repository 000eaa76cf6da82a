"""Philox4x32-10 and the 53-bit uniform draw (oracle copy, pure Python).

Philox4x32 is defined in J. K. Salmon, M. A. Moraes, R. O. Dror and D. E. Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11: a 10-round
substitution-permutation network on a 128-bit counter with a 64-bit key.
Each round multiplies counter words 0 and 2 by two fixed 32-bit multipliers,
mixes the high halves with the other two words and the round key, and the key
is advanced by two Weyl constants between rounds.

Both samplers draw their randomness from this generator so that a given
(seed, sample, operation) triple gives the same number on the CPU and the GPU.
The paper does not fix a generator or a draw rule; this one is a reading of
the paper, the same on both sides.
"""
from __future__ import annotations

MASK32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85

PURPOSE_UPDATE = 0   # draw for UpdateState (Alg. 1)
PURPOSE_KRAUS = 1    # draw of the Kraus index (Eq. 5)


def philox4x32_10(ctr, key):
    """Ten Philox rounds on counter (c0,c1,c2,c3) with key (k0,k1)."""
    c0, c1, c2, c3 = (int(v) & MASK32 for v in ctr)
    k0, k1 = (int(v) & MASK32 for v in key)
    for r in range(10):
        if r:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
    return c0, c1, c2, c3


def uniform53(w0: int, w1: int) -> float:
    """A double in [0,1) from the top 27 bits of w0 and the top 26 bits of w1."""
    return ((w0 >> 5) * 67108864.0 + (w1 >> 6)) * (1.0 / 9007199254740992.0)


def draw(seed: int, sample_id: int, op_id: int, purpose: int) -> float:
    """The uniform used at operation ``op_id`` of sample ``sample_id``.

    key = (seed lo, seed hi); counter = (sample lo, sample hi, op_id, purpose).
    """
    w = philox4x32_10((sample_id & MASK32, (sample_id >> 32) & MASK32, op_id, purpose),
                      (seed & MASK32, (seed >> 32) & MASK32))
    return uniform53(w[0], w[1])
