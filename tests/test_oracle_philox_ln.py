"""Pins for the oracle's Philox-4x32-10 and its ln (no GPU)."""
import math
import os
import struct

import numpy as np
import pytest

import oracle


def _kat():
    # known-answer vectors published with Philox (fixture cites the source)
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    out = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out.append((w[0:4], w[4:6], w[6:10]))
    return out


KAT = _kat()


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


def _f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def _ulp_diff(a, b):
    ia = struct.unpack("<i", struct.pack("<f", a))[0]
    ib = struct.unpack("<i", struct.pack("<f", b))[0]
    return abs(ia - ib)


def test_ln_against_libm():
    # the UCT logarithm works in IEEE single precision: within 1 ulp of the
    # correctly rounded libm value at every visit count tried
    xs = list(range(1, 20000)) + [int(v) for v in np.geomspace(20000, 4e9, 5000)]
    worst = max(_ulp_diff(oracle.lnf(_f32(float(x))), _f32(math.log(_f32(float(x))))) for x in xs if x > 1)
    assert oracle.lnf(1.0) == 0.0
    assert worst <= 1, worst


def test_ln_reduction_boundaries():
    # both sides of the sqrt(2) switch of the mantissa, powers of two, large counts
    for x in [math.sqrt(2.0), 1.4142135, 1.4142137, 2.0 * math.sqrt(2.0), 2.0, 4.0, 3.0, 1.5, 1e6 + 1.0,
              2.0 ** 40 + 7]:
        xf = _f32(x)
        assert _ulp_diff(oracle.lnf(xf), _f32(math.log(xf))) <= 1, x
