"""Pins of the oracle's random-number streams.

Philox4x32-10 is pinned by the published known-answer vectors; the
Box-Muller normals by their moments and a Kolmogorov-Smirnov test against the
standard normal CDF (scipy); the four-normals-per-draw indexing by recomputing
one stream from raw Philox words.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        assert f[0] == "10"
        v = [int(x, 16) for x in f[1:]]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle):
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert oracle.philox4x32_10(ctr, key) == want


def test_philox_counter_sensitivity(oracle):
    # every counter and key word changes every output word (avalanche)
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        ctr = [1, 2, 3, 4]
        ctr[i] ^= 1
        out = oracle.philox4x32_10(ctr, [5, 6])
        assert all(a != b for a, b in zip(out, base))
    out = oracle.philox4x32_10([1, 2, 3, 4], [5, 7])
    assert all(a != b for a, b in zip(out, base))


def test_box_muller_special_values(oracle):
    # u2 = 1/2 - 2^-33 puts the angle just below pi: z0 ~ -r, z1 ~ +0
    z0, z1 = oracle.box_muller(0x7FFFFFFF, 0x7FFFFFFF)
    u1 = (0x7FFFFFFF + 0.5) / 2**32
    r = math.sqrt(-2.0 * math.log(u1))
    assert z0 == pytest.approx(-r, rel=1e-12)
    assert abs(z1) < 1e-8
    # smallest u1 gives the largest radius, sqrt(2*(33 ln 2 + ln 1/1)) region
    z0, z1 = oracle.box_muller(0, 0)
    assert math.hypot(z0, z1) == pytest.approx(math.sqrt(-2 * math.log(0.5 / 2**32)), rel=1e-12)
    # radius is independent of u2
    a = oracle.box_muller(12345, 1)
    b = oracle.box_muller(12345, 3_000_000_000)
    assert math.hypot(*a) == pytest.approx(math.hypot(*b), rel=1e-12)


def test_normals_are_standard(oracle):
    n = 40000
    z = np.array([oracle.normal(7, oracle.TAG_MUT, 3, 11, j) for j in range(n)])
    assert abs(z.mean()) < 4.0 / math.sqrt(n)
    assert abs(z.std() - 1.0) < 4.0 * math.sqrt(0.5 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # pairs are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 4.0 / math.sqrt(n / 2)


def test_normal_indexing_four_per_draw(oracle):
    # normal j is member j%4 of the draw {j/4, t, tag, id}: (0,1) cos/sin of
    # lanes (0,1), (2,3) cos/sin of lanes (2,3)
    seed, tag, t, ident = 0x123456789ABCDEF, oracle.TAG_INIT_W, 0, 17
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for q in (0, 1, 5832):
        r = oracle.philox4x32_10([q, t, tag, ident], key)
        want = list(oracle.box_muller(r[0], r[1])) + list(oracle.box_muller(r[2], r[3]))
        got = [oracle.normal(seed, tag, t, ident, 4 * q + i) for i in range(4)]
        assert got == want
