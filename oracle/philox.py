"""Philox4x32-10 counter-based generator and the sampler's draw contract.

Philox4x32-10 follows Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplies
with the Weyl key schedule. Written from the published definition.

Draw contract (identical on the CUDA side, implemented there separately):

* key = (seed mod 2^32, seed >> 32)
* measurement event e of shot s draws u in [0, 1) on the 53-bit grid,
  u = (T * 2^52 + L) * 2^-53, where
  - T = bit (s mod 128) of the block draw Philox(key, (g lo, g hi, TAG_MT, e)),
    g = s >> 7; bit b of a 128-bit output is bit (b mod 32) of word b / 32;
  - L = low 52 bits of w0 | w1 << 32 of Philox(key, (s lo, s hi, TAG_ML, e)).
  The outcome is m = [u < P(m = 1)].
* gap draw of shot s that starts its search at site index ``start``:
  Philox(key, (s lo, s hi, TAG_GAP, start)); w0 | w1 << 32 is the 64-bit
  uniform for the survival search, w2 picks the fault's Pauli option.
"""

from __future__ import annotations

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

TAG_MT = 1    # measurement, top bit (per 128-shot block)
TAG_ML = 2    # measurement, low 52 bits (per shot)
TAG_GAP = 3   # noise gap draw (per shot)


def philox4x32_10(ctr: tuple[int, int, int, int], key: tuple[int, int]) -> tuple[int, int, int, int]:
    c0, c1, c2, c3 = (x & MASK32 for x in ctr)
    k0, k1 = (x & MASK32 for x in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def key_of(seed: int) -> tuple[int, int]:
    return seed & MASK32, (seed >> 32) & MASK32


def meas_u(seed: int, shot: int, event: int) -> float:
    """The uniform u of measurement event ``event`` in shot ``shot``."""
    key = key_of(seed)
    g = shot >> 7
    blk = philox4x32_10((g & MASK32, g >> 32, TAG_MT, event), key)
    b = shot & 127
    top = (blk[b >> 5] >> (b & 31)) & 1
    w = philox4x32_10((shot & MASK32, shot >> 32, TAG_ML, event), key)
    low = (w[0] | (w[1] << 32)) & ((1 << 52) - 1)
    return ((top << 52) | low) * 2.0 ** -53


def meas_top_bit(seed: int, shot: int, event: int) -> int:
    key = key_of(seed)
    g = shot >> 7
    blk = philox4x32_10((g & MASK32, g >> 32, TAG_MT, event), key)
    b = shot & 127
    return (blk[b >> 5] >> (b & 31)) & 1


def gap_draw(seed: int, shot: int, start: int) -> tuple[int, int]:
    """(64-bit uniform for the survival search, 32-bit option word)."""
    w = philox4x32_10((shot & MASK32, shot >> 32, TAG_GAP, start), key_of(seed))
    return w[0] | (w[1] << 32), w[2]
