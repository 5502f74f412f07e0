"""Counter-based Philox generators (oracle side).

Test infrastructure only: nothing in the product path imports this module.

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of a
multiply-high/low Feistel-like bijection of a 128-bit counter under a 64-bit
key, with the key bumped by two Weyl constants between rounds.  The paper under
study draws its errors with external samplers (Sec. "Numerical Results"); the
counter-based form here makes every shot reproducible on its own, which is what
lets the CUDA sampler be checked bit for bit.

`philox4x64_10` is the same construction with 64-bit words; it exists only so
that a test can compare the round structure with `numpy.random.Philox`, an
independent implementation of that variant.
"""
import numpy as np

M4x32_0 = 0xD2511F53
M4x32_1 = 0xCD9E8D57
W32_0 = 0x9E3779B9
W32_1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)

M4x64_0 = 0xD2E7470EE14C6C93
M4x64_1 = 0xCA5A826395121157
W64_0 = 0x9E3779B97F4A7C15
W64_1 = 0xBB67AE8584CAA73B
_MASK64 = (1 << 64) - 1


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds, vectorised over numpy arrays of 32-bit words.

    Every argument is an integer array (or scalar) holding values below 2**32;
    they broadcast against each other.  Returns four uint64 arrays holding the
    32-bit output words.
    """
    c0 = np.asarray(c0, dtype=np.uint64)
    c1 = np.asarray(c1, dtype=np.uint64)
    c2 = np.asarray(c2, dtype=np.uint64)
    c3 = np.asarray(c3, dtype=np.uint64)
    k0 = np.asarray(k0, dtype=np.uint64)
    k1 = np.asarray(k1, dtype=np.uint64)
    m0 = np.uint64(M4x32_0)
    m1 = np.uint64(M4x32_1)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(W32_0)) & _MASK32
            k1 = (k1 + np.uint64(W32_1)) & _MASK32
        p0 = m0 * c0  # < 2**64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def philox4x64_10(ctr, key):
    """Ten Philox4x64 rounds on Python integers (4 counter words, 2 key words)."""
    c = list(ctr)
    k = list(key)
    for rnd in range(10):
        if rnd > 0:
            k = [(k[0] + W64_0) & _MASK64, (k[1] + W64_1) & _MASK64]
        p0 = M4x64_0 * c[0]
        p1 = M4x64_1 * c[2]
        hi0, lo0 = p0 >> 64, p0 & _MASK64
        hi1, lo1 = p1 >> 64, p1 & _MASK64
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
    return c


def unit_words(shots, n_units, seed, stream=0):
    """The 32-bit draw of every (shot, unit) pair.

    Counter = (shot low word, shot high word, unit >> 2, stream), key =
    (seed low word, seed high word); unit u takes output word u & 3.  `shots`
    is an array of global shot indices.  Returns a uint64 array of shape
    (len(shots), n_units).
    """
    shots = np.asarray(shots, dtype=np.uint64)
    seed = int(seed)
    n_blocks = (n_units + 3) // 4
    blk = np.arange(n_blocks, dtype=np.uint64)[None, :]
    s_lo = (shots & _MASK32)[:, None]
    s_hi = (shots >> np.uint64(32))[:, None]
    out = philox4x32_10(s_lo, s_hi, blk, np.uint64(stream),
                        np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    words = np.stack(out, axis=-1).reshape(len(shots), n_blocks * 4)
    return words[:, :n_units]
