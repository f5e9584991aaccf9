"""Philox4x32-10 counter-based generator (oracle side; test use only).

Written from its published definition (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11): a 4 x 32-bit counter, a
2 x 32-bit key, ten rounds of two 32x32->64 multiplications, with the key
bumped by the Weyl constants between rounds.  The GA draws (§4.2, §5) are
taken from it so that the GPU and the oracle see the same random numbers.

Pinned by the known-answer vectors published with that paper's reference
implementation (tests/golden/philox4x32_10_kat.txt).
"""
from __future__ import annotations

MASK = 0xFFFFFFFF
MUL0, MUL1 = 0xD2511F53, 0xCD9E8D57
WEYL0, WEYL1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr, key):
    c0, c1, c2, c3 = (int(x) & MASK for x in ctr)
    k0, k1 = (int(x) & MASK for x in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + WEYL0) & MASK
            k1 = (k1 + WEYL1) & MASK
        prod0 = MUL0 * c0
        prod1 = MUL1 * c2
        c0, c1, c2, c3 = ((prod1 >> 32) ^ c1 ^ k0) & MASK, prod1 & MASK, \
                         ((prod0 >> 32) ^ c3 ^ k1) & MASK, prod0 & MASK
    return c0, c1, c2, c3


# Draw streams of the GA.  A stream is identified by (seed, generation g,
# chromosome q, operator t); its words are block d = 0, 1, 2, ... of
# philox4x32_10(counter = (g, q, t, d), key = (seed lo, seed hi)), each block
# read w0, w1, w2, w3 in order.
OP_PERTURB, OP_CROSSOVER, OP_CORRECTION, OP_MUTATION = 0, 1, 2, 3


class DrawStream:
    def __init__(self, seed: int, g: int, q: int, t: int):
        self.key = (seed & MASK, (seed >> 32) & MASK)
        self.g, self.q, self.t = g, q, t
        self.block = 0
        self.buf = []

    def word(self) -> int:
        if not self.buf:
            self.buf = list(philox4x32_10((self.g, self.q, self.t, self.block), self.key))
            self.block += 1
        return self.buf.pop(0)

    def below(self, m: int) -> int:
        """An integer in [0, m): the high half of the 64-bit product word * m."""
        return (self.word() * m) >> 32
