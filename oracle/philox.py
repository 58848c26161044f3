"""Philox4x32-10 counter-based random numbers (oracle side; test infrastructure).

Definition: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11.  A 128-bit counter (four 32-bit words) is
mixed with a 64-bit key (two words) by ten rounds.  Each round multiplies
words 0 and 2 by fixed odd constants, splits the 64-bit products into high and
low halves, and permutes/XORs them with words 1, 3 and the round key.  The key
is advanced by two Weyl constants between rounds.

The paper draws prior samples and noise with torch's RNG on the GPU (Sec. 3.2).
Here both the oracle and the GPU path implement this one published generator,
so that the same (seed, counter) gives the same integers on both sides.

Stream layout used by the method (the GPU library implements the same):
counter = (index, block, tag, step), key = (seed & 0xffffffff, seed >> 32).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

TAG_PRIOR = 1   # parameter draws (one counter per draw)
TAG_NOISE = 2   # background noise (one counter per pair of frequency bins)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds over broadcastable uint32 arrays; returns four uint32 arrays."""
    c = [np.asarray(x, dtype=np.uint32) for x in np.broadcast_arrays(c0, c1, c2, c3)]
    k0 = np.asarray(k0, dtype=np.uint32)
    k1 = np.asarray(k1, dtype=np.uint32)
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = (k0 + W0).astype(np.uint32)
                k1 = (k1 + W1).astype(np.uint32)
            p0 = M0 * c[0].astype(np.uint64)
            p1 = M1 * c[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & MASK32).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def key_of(seed):
    """Split a 64-bit seed into the two key words."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint32(seed & 0xFFFFFFFF), np.uint32(seed >> 32)


def uniform52(w_hi, w_lo):
    """Uniform double in (0, 1) from two words: (x + 1/2) 2^-52 with x the top 52 bits.

    x + 1/2 needs 53 significant bits, so the value is exact in binary64 and the
    GPU path, which uses the same formula, produces the identical double.
    """
    x = (np.asarray(w_hi, dtype=np.uint64) << np.uint64(20)) | (
        np.asarray(w_lo, dtype=np.uint64) >> np.uint64(12))
    return (x.astype(np.float64) + 0.5) * 2.0 ** -52


def uniform24(w):
    """Uniform in (0, 1) on a 2^-24 grid: ((w >> 8) + 1/2) 2^-24, exact in binary32 and binary64."""
    x = np.asarray(w, dtype=np.uint32) >> np.uint32(8)
    return (x.astype(np.float64) + 0.5) * 2.0 ** -24


def bounded_index(w, n):
    """Integer in [0, n) from one word by multiply-shift: floor(w * n / 2^32) (n < 2^32)."""
    return ((np.asarray(w, dtype=np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
