"""Philox4x32-10 counter-based generator, FP64 oracle side.

TEST INFRASTRUCTURE: this module belongs to the CPU oracle. Only tests, the
smoke check and the CPU-baseline leg of the benchmark may import it.

The paper draws its measurement matrix C from i.i.d. random samples
(Algorithm 1 step 2; Section 3.3 "Measurement Matrices") and notes that the
random draws parallelise well on a GPU (Section 3.4).  It does not name a
generator.  We use Philox4x32-10 from Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 4-word counter and a
2-word key go through ten rounds; each round multiplies words 0 and 2 by two
fixed odd constants, forms the output words from the high/low halves of those
products xor-ed with the other two words and the round key, and the key is
bumped by two Weyl constants between rounds.

Written from that definition with numpy uint64 arithmetic (32x32->64 bit
products are exact in uint64).  Vectorised over counters; no blocking.
"""
import numpy as np

# Multipliers and Weyl key increments of Philox4x32 (Salmon et al., SC'11).
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
PHILOX_ROUNDS = 10

_MASK32 = np.uint64(0xFFFFFFFF)
_SHIFT32 = np.uint64(32)


def philox4x32_10(ctr, key):
    """Apply the ten-round Philox4x32 bijection.

    ctr: array (..., 4) of uint32 counters; key: (k0, k1) python ints.
    Returns an array (..., 4) uint32 of output words.
    """
    c = np.asarray(ctr, dtype=np.uint64)
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    for rnd in range(PHILOX_ROUNDS):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
            k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
        p0 = PHILOX_M0 * c0          # exact: both factors < 2^32
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> _SHIFT32, p0 & _MASK32
        hi1, lo1 = p1 >> _SHIFT32, p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def seed_key(seed):
    """Split a 64-bit seed into the Philox key (low word, high word)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)
