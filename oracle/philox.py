"""Philox4x32-10 and the xi-sampling map (oracle side; test infrastructure only).

Philox4x32-10 is written from its published definition (J. K. Salmon,
M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11, Sec. 3.3): a 4-word, 32-bit-per-word counter is passed through
10 rounds; each round multiplies words 0 and 2 by two fixed constants, keeps
the high and low halves of the 64-bit products, and XORs the high halves into
the other two words together with that round's key.  The 2-word key advances
by the Weyl increments (golden ratio and sqrt(3)-1 in 32-bit fixed point)
between rounds.  Pure Python integers: slow, exact, obviously 32-bit.

The paper samples xi_1, xi_2, xi_3 independently and uniformly on [-1, 1]
(Sec. 4, the paragraph on porosity and recharge).  Map used here, exact in
binary64: take 52 bits u = (w0 << 20) | (w1 >> 12) from two words, form the
odd integer k = 2u + 1 - 2^52 (|k| < 2^52) and return k * 2^-52, which lies in
(-1, 1) and is symmetric about 0.

Counter layout per sample s at MLMC level l (key = the two 32-bit halves of
the 64-bit seed): block 0 = (l, lo32(s), hi32(s), 0) gives xi_1 from words
(0, 1) and xi_2 from words (2, 3); block 1 = (l, lo32(s), hi32(s), 1) gives
xi_3 from words (0, 1).
"""
import numpy as np

MASK32 = 0xFFFFFFFF
# Round multipliers and key increments of Philox4x32 (SC'11, Table 2 and Sec. 3.3).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85


def philox4x32_10(ctr, key):
    """Return the 4 output words of Philox4x32 with 10 rounds for counter
    ``ctr`` (4 ints < 2^32) and key ``key`` (2 ints < 2^32)."""
    x0, x1, x2, x3 = (int(v) & MASK32 for v in ctr)
    k0, k1 = (int(v) & MASK32 for v in key)
    for rnd in range(10):
        if rnd > 0:  # key schedule: bump before every round but the first
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * x0
        p1 = PHILOX_M1 * x2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        x0, x1, x2, x3 = (hi1 ^ x1 ^ k0) & MASK32, lo1, (hi0 ^ x3 ^ k1) & MASK32, lo0
    return x0, x1, x2, x3


def words_to_unit(w_hi, w_lo):
    """Map two 32-bit words to a float in (-1, 1) exactly: 52 random bits u,
    odd integer k = 2u + 1 - 2^52, value k / 2^52."""
    u = ((int(w_hi) & MASK32) << 20) | ((int(w_lo) & MASK32) >> 12)
    k = 2 * u + 1 - (1 << 52)
    return float(k) * 2.0 ** -52  # |k| < 2^53: the conversion is exact


def sample_xi(seed, level, first_sample, n, n_xi=3):
    """xi[n][n_xi] for samples first_sample .. first_sample+n-1 of ``level``."""
    key = (seed & MASK32, (seed >> 32) & MASK32)
    out = np.empty((n, n_xi), dtype=np.float64)
    for i in range(n):
        s = first_sample + i
        vals = []
        blk = 0
        while len(vals) < n_xi:
            w = philox4x32_10((level, s & MASK32, (s >> 32) & MASK32, blk), key)
            vals.append(words_to_unit(w[0], w[1]))
            if len(vals) < n_xi:
                vals.append(words_to_unit(w[2], w[3]))
            blk += 1
        out[i] = vals[:n_xi]
    return out
