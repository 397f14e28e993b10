"""Pins for the oracle's Philox-4x32-10 and its ln (no GPU)."""
import math
import struct

import numpy as np
import pytest

import oracle


# Known-answer vectors published with Philox (Salmon et al., SC'11, Random123
# distribution, kat_vectors: philox4x32 with 10 rounds).
KAT = [
    ([0x00000000, 0x00000000, 0x00000000, 0x00000000], [0x00000000, 0x00000000],
     [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF], [0xFFFFFFFF, 0xFFFFFFFF],
     [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
]


@pytest.mark.parametrize("ctr,key,want", KAT)
def test_philox_known_answers(ctr, key, want):
    assert oracle.philox4x32_10(ctr, key) == want


def test_philox_words_uniform():
    # 4 * 20000 words into 16 bins of the top nibble: chi-square sanity check.
    from scipy.stats import chisquare
    words = []
    for k in range(20000):
        words += oracle.philox4x32_10([k, 7, 11, 2], [12345, 678])
    bins = np.bincount(np.array(words, dtype=np.uint64) >> np.uint64(28), minlength=16)
    assert chisquare(bins).pvalue > 1e-4


def _ulp_diff(a, b):
    ia = struct.unpack("<q", struct.pack("<d", a))[0]
    ib = struct.unpack("<q", struct.pack("<d", b))[0]
    return abs(ia - ib)


def test_ln_against_libm():
    xs = list(range(1, 5000)) + [int(v) for v in np.geomspace(5000, 4e9, 3000)]
    worst = max(_ulp_diff(oracle.ln(float(x)), math.log(float(x))) for x in xs if x > 1)
    assert oracle.ln(1.0) == 0.0
    assert worst <= 2, worst


def test_ln_reduction_boundaries():
    for x in [math.sqrt(2.0), 2.0 * math.sqrt(2.0), 3.0, 1.5, 1e6 + 1.0, 2.0 ** 40 + 7]:
        assert abs(oracle.ln(x) - math.log(x)) <= 4e-16 * max(1.0, abs(math.log(x)))
