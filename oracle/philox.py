"""Philox4x32-10 counter-based generator and the draws the Squint update takes.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this module.

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel Random Numbers: As Easy as 1, 2, 3", SC'11, Section 3.2): a 4x32-bit
counter and a 2x32-bit key, ten rounds of two 32x32->64 multiplies whose high
halves are xored with the other two words and the round key, the key bumped by
the two Weyl constants between rounds.

The paper on Squint (Algorithm 1) draws a minibatch, random shifts and the
reparameterisation noise of the tanh-Gaussian actor, without saying how.  The
reading used on both sides of the parity tests: every draw is one Philox block
addressed by (element, stream | sub_block << 16, word_lo, word_hi) under key
(seed_lo, seed_hi), where (word_lo, word_hi) is the 64-bit update index (update
draws), the tensor id (weight init) or the request key (actor inference).
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

# Stream ids (the second counter word, low 16 bits).
STREAM_INDEX = 1        # minibatch slot indices
STREAM_SHIFT_T = 2      # random shift of o_t
STREAM_SHIFT_T1 = 3     # random shift of o_{t+1}
STREAM_EPS_TARGET = 4   # actor noise at s_{t+1} (target)
STREAM_EPS_ACTOR = 5    # actor noise at s_t (alpha and actor losses)
STREAM_INIT = 16        # parameter initialisation
STREAM_ACT = 32         # actor noise for inference requests


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on arrays of 32-bit words; returns four uint64 arrays < 2**32."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & MASK32)
    k1 = np.uint64(int(k1) & MASK32)
    m0, m1 = np.uint64(M0), np.uint64(M1)
    for rnd in range(10):
        p0 = m0 * c0                      # < 2**64, exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK32)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if rnd < 9:
            k0 = np.uint64((int(k0) + W0) & MASK32)
            k1 = np.uint64((int(k1) + W1) & MASK32)
    return c0, c1, c2, c3


def block(seed, element, stream, word, sub=0):
    """Philox block for draw `element` of `stream`, addressed by a 64-bit `word`."""
    element = np.asarray(element, dtype=np.uint64)
    word = int(word)
    c1 = np.full(element.shape, (stream & 0xFFFF) | ((sub & 0xFFFF) << 16), dtype=np.uint64)
    c2 = np.full(element.shape, word & MASK32, dtype=np.uint64)
    c3 = np.full(element.shape, (word >> 32) & MASK32, dtype=np.uint64)
    seed = int(seed)
    return philox4x32_10(element, c1, c2, c3, seed & MASK32, (seed >> 32) & MASK32)


def mulhi_range(w, n):
    """floor(w * n / 2**32): an integer in [0, n) from a 32-bit word (multiply-shift)."""
    return ((np.asarray(w, dtype=np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def uniform01(w):
    """Open-interval uniform from the top 23 bits of a word: ((w >> 9) + 0.5) / 2**23.

    23 bits keep (w >> 9) + 0.5 exact in FP32 as well as FP64, so both precisions
    see the same uniform value.
    """
    return ((np.asarray(w, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def normal_pairs(seed, stream, word, rows, dim):
    """Standard normals eps[rows, dim] by Box-Muller: pair q of row b uses block (b, stream, word, q)."""
    b = np.arange(rows, dtype=np.uint64)
    eps = np.empty((rows, dim), dtype=np.float64)
    for q in range((dim + 1) // 2):
        w = block(seed, b, stream, word, sub=q)
        u1, u2 = uniform01(w[0]), uniform01(w[1])
        rad = np.sqrt(-2.0 * np.log(u1))
        ang = 2.0 * np.pi * u2
        eps[:, 2 * q] = rad * np.cos(ang)
        if 2 * q + 1 < dim:
            eps[:, 2 * q + 1] = rad * np.sin(ang)
    return eps
