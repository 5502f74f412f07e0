"""Pins for the oracle's Philox generator and its (shot, unit) word layout."""
import numpy as np
import pytest

from oracle import philox
from oracle.sampler import pauli_thresholds


# Known-answer vectors published with the Random123 reference implementation of
# Philox4x32-10 (counter words, key words) -> output words.
KAT_4X32 = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,want", KAT_4X32)
def test_philox4x32_known_answers(ctr, key, want):
    got = philox.philox4x32_10(*ctr, *key)
    assert tuple(int(x) for x in got) == want


def test_philox4x64_matches_numpy():
    # numpy.random.Philox is an independent implementation of the 4x64-10 variant; it
    # increments its counter before each block, so block b uses counter b + 1.
    for key in ([0, 0], [12345, 678], [2**64 - 1, 3]):
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.zeros(4, dtype=np.uint64))
        raw = [int(x) for x in bg.random_raw(12)]
        for b in range(3):
            mine = philox.philox4x64_10([b + 1, 0, 0, 0], key)
            assert mine == raw[4 * b:4 * b + 4]


def test_unit_word_layout():
    shots = np.array([0, 1, 2**32 + 5])
    words = philox.unit_words(shots, 10, seed=(7 << 32) | 9, stream=3)
    for si, shot in enumerate(shots):
        for u in range(10):
            blk = philox.philox4x32_10(int(shot) & 0xFFFFFFFF, int(shot) >> 32, u >> 2, 3, 9, 7)
            assert int(words[si, u]) == int(blk[u & 3])


def test_pauli_frequencies_within_5_sigma():
    p = 0.12
    n_shots = 4000
    u = philox.unit_words(np.arange(n_shots), 25, seed=11)
    t1, t2, t3 = pauli_thresholds(p)
    n = u.size
    for lo, hi in ((0, t1), (t1, t2), (t2, t3)):
        freq = np.count_nonzero((u >= lo) & (u < hi))
        mean = n * p / 3
        assert abs(freq - mean) < 5 * np.sqrt(mean * (1 - p / 3))
