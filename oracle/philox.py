"""Counter-based Gaussian draws for the oracle (test infrastructure only).

The paper draws a fresh standard Gaussian vector g_t at every step (Algorithm 1 and
Algorithm 2; Section 3.2 requires each new draw to be independent of everything built
so far) but fixes no generator.  Both implementations therefore follow one published
counter-based generator, Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), so that a draw is a pure function
of (seed, trial, step, stream, index).  This module is the oracle's own copy, written
in plain numpy from that definition; it shares nothing with the CUDA path.

Layout of one draw (index i of a stream, 0-based):
  * Philox key   = (seed mod 2^32, seed >> 32)
  * Philox block = (i >> 1, step, trial, stream)  -> four 32-bit words (w0, w1, w2, w3)
  * u1 = (((w0 << 21) | (w1 >> 11)) + 1) * 2^-53,   u2 likewise from (w2, w3); u in (0, 1]
  * Box-Muller: r = sqrt(-2 ln u1); index 2j gets r cos(2 pi u2), index 2j+1 gets
    r sin(2 pi u2).
Indices a step does not use (the masked head of Algorithm 1, the entries g_t[1:t-1]
that H_t(g_t) ignores in Algorithm 2) are never drawn; skipping them gives the same
values as drawing and discarding them, because every index has its own counter.
"""
import numpy as np

# Philox4x32 multipliers and Weyl key increments (Salmon et al., SC'11, Section 4).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
PHILOX_ROUNDS = 10

MASK32 = np.uint64(0xFFFFFFFF)

STREAM_G = 0  # the Gaussian vectors g_t of the algorithm


def philox4x32(c0, c1, c2, c3, seed, rounds=PHILOX_ROUNDS):
    """Philox4x32-`rounds` on arrays of 32-bit counters; returns four uint64 arrays of words.

    One round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 as 64-bit products, then
    (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by
    the Weyl constants between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    k0 = seed & 0xFFFFFFFF
    k1 = seed >> 32
    for _ in range(rounds):
        p0 = c0 * np.uint64(PHILOX_M0)          # < 2^64, exact in uint64
        p1 = c2 * np.uint64(PHILOX_M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
        k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
    return c0, c1, c2, c3


def uniform53(hi_word, lo_word):
    """Map two 32-bit words to a double in (0, 1]: (53-bit integer + 1) * 2^-53 (exact)."""
    k = (np.asarray(hi_word, dtype=np.uint64) << np.uint64(21)) | (
        np.asarray(lo_word, dtype=np.uint64) >> np.uint64(11))
    return (k.astype(np.float64) + 1.0) * 2.0 ** -53


def normals(seed, trial, step, start, count, stream=STREAM_G):
    """Standard normals for absolute indices start..start+count-1 of (seed, trial, step, stream)."""
    if count <= 0:
        return np.zeros(0, dtype=np.float64)
    idx = np.arange(start, start + count, dtype=np.int64)
    j0, j1 = int(idx[0] >> 1), int(idx[-1] >> 1)
    pairs = np.arange(j0, j1 + 1, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32(pairs, step, trial, stream, seed)
    u1 = uniform53(w0, w1)
    u2 = uniform53(w2, w3)
    r = np.sqrt(-2.0 * np.log(u1))
    theta = 2.0 * np.pi * u2
    both = np.empty(2 * len(pairs), dtype=np.float64)
    both[0::2] = r * np.cos(theta)
    both[1::2] = r * np.sin(theta)
    off = start - 2 * j0
    return both[off:off + count]


def gaussian_vector(seed, trial, step, dim, first, sigma=1.0, stream=STREAM_G):
    """g in R^dim with entries sigma*N(0,1) at 0-based indices first..dim-1 and zeros before.

    This is Z_{1:first} g in the paper's notation (indices 1..first masked), used for the
    draws of Algorithms 1 and 2.
    """
    g = np.zeros(dim, dtype=np.float64)
    if first < dim:
        g[first:] = sigma * normals(seed, trial, step, first, dim - first, stream)
    return g
