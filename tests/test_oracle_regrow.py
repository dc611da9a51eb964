"""Pins of the oracle's regrowth (App. B.1, Eq. (1)).

* bit-exact reconstruction: neighbour counts by 2-D convolution (scipy),
  count classes by comparison with the class edges, Philox words from an
  independent numpy Philox; any wrong radius, shape, class edge, row index,
  counter layout or a non-synchronous update fails it;
* per (row, class) growth frequencies over many steps against the closed
  form p = p_I c(row) + c within a binomial bound;
* invariants: no growth where the count is zero unless spontaneous growth is
  on, no growth at all when every probability is zero, walls never grow,
  resources never vanish during regrowth.
"""
import math

import numpy as np
import pytest
from scipy import signal, stats

from paper_2302_09334_gb300.params import EcoParams
from tests import philox_np


def test_philox_np_known_answers(oracle):
    from tests.test_oracle_rng import _kat_rows
    for ctr, key, want in _kat_rows():
        got = philox_np.philox(*[np.uint32(c) for c in ctr], key[0], key[1])
        assert [int(g) for g in got] == want


def _kernel(shape, radius):
    r = radius
    dy, dx = np.mgrid[-r:r + 1, -r:r + 1]
    if shape == 1:
        k = (np.abs(dy) + np.abs(dx) <= r)
    else:
        k = np.ones_like(dy, bool)
    k[r, r] = False
    return k.astype(np.int64)


def _reconstruct(p: EcoParams, seed, t, res, wall, thr):
    counts = signal.convolve2d(res.astype(np.int64), _kernel(p.nbr_shape, p.nbr_radius),
                               mode="same", boundary="fill", fillvalue=0)
    cls = (counts[..., None] >= np.array(p.class_edges)[None, None, :]).sum(-1)
    u = philox_np.grid_words(seed, p.H, p.W, t, 1)
    rows = np.arange(p.H)[:, None].repeat(p.W, 1)
    grow = u < thr[rows, cls]
    empty = (res == 0) & (wall == 0)
    return np.where(empty, grow, res).astype(np.uint8)


@pytest.mark.parametrize("shape,radius", [(0, 2), (0, 1), (1, 1), (1, 3), (0, 3)])
def test_regrow_bit_exact_reconstruction(oracle, shape, radius):
    p = EcoParams(H=37, W=70, nbr_shape=shape, nbr_radius=radius,
                  p_class=(0.0, 0.05, 0.2, 0.6), p_spont=0.01, border_walls=1)
    rng = np.random.default_rng(1)
    wall = np.zeros((p.H, p.W), np.uint8)
    wall[0, :] = wall[-1, :] = wall[:, 0] = wall[:, -1] = 1
    wall[rng.random((p.H, p.W)) < 0.03] = 1
    res = ((rng.random((p.H, p.W)) < 0.2) & (wall == 0)).astype(np.uint8)
    thr = oracle.threshold_table(p.asdict())
    for t in (0, 1, 77, 2**31 + 5):
        got = oracle.regrow(p.asdict(), 99, t, res, wall, thr)
        want = _reconstruct(p, 99, t, res, wall, thr)
        np.testing.assert_array_equal(got, want)


def test_threshold_rows_and_direction(oracle):
    p = EcoParams(H=11, W=8)
    thr = oracle.threshold_table(p.asdict()).astype(np.float64) / 2**32
    # class 0 is spontaneous growth only, identical on every row
    assert np.all(thr[:, 0] == thr[0, 0])
    assert thr[0, 0] == pytest.approx(p.p_spont, abs=2**-32)
    # the latitude factor rises from lat_top (top row) to lat_bottom (bottom)
    for cls in (1, 2, 3):
        assert np.all(np.diff(thr[:, cls]) > 0)
        assert thr[0, cls] == pytest.approx(p.p_class[cls] * p.lat_top + p.p_spont, abs=2**-31)
        assert thr[-1, cls] == pytest.approx(p.p_class[cls] * p.lat_bottom + p.p_spont, abs=2**-31)
    # paper form c(x) = (alpha^x + 1) / (alpha + 1): from 2/(alpha+1) to 1
    q = p.replace(lat_mode=1, p_spont=0.0)
    thr = oracle.threshold_table(q.asdict()).astype(np.float64) / 2**32
    assert thr[0, 3] == pytest.approx(0.025 * 2 / 201, abs=2**-32)
    assert thr[-1, 3] == pytest.approx(0.025, abs=2**-32)
    # probabilities of one or more saturate at the largest threshold
    q = p.replace(p_class=(0.0, 0.5, 1.0, 7.0), lat_top=1.0, lat_bottom=1.0, p_spont=0.0)
    thr = oracle.threshold_table(q.asdict())
    assert thr[0, 1] == 2**31 and thr[0, 2] == 0xFFFFFFFF and thr[0, 3] == 0xFFFFFFFF
    assert thr[0, 0] == 0


def test_regrow_frequencies_match_closed_form(oracle):
    p = EcoParams(H=24, W=64, border_walls=0, p_class=(0.0, 0.1, 0.2, 0.3), p_spont=0.02)
    rng = np.random.default_rng(5)
    res = (rng.random((p.H, p.W)) < 0.15).astype(np.uint8)
    wall = np.zeros_like(res)
    counts = signal.convolve2d(res.astype(np.int64), _kernel(0, 2), mode="same")
    cls = np.searchsorted(np.array([1, 3, 5]), counts, side="right")
    empty = res == 0
    thr = oracle.threshold_table(p.asdict())
    M = 300
    grown = np.zeros((p.H, p.W), np.int64)
    for t in range(M):
        grown += oracle.regrow(p.asdict(), 2024, t, res, wall, thr) & empty
    n_groups = 0
    for y in range(p.H):
        lat = p.lat_top + (p.lat_bottom - p.lat_top) * y / (p.H - 1)
        for c in range(4):
            sel = empty[y] & (cls[y] == c)
            n = int(sel.sum()) * M
            if n == 0:
                continue
            k = int(grown[y][sel].sum())
            prob = p.p_class[c] * lat + p.p_spont
            n_groups += 1
            assert stats.binomtest(k, n, prob).pvalue > 1e-4, (y, c, k, n, prob)
    assert n_groups > 60


def test_regrow_invariants(oracle):
    rng = np.random.default_rng(9)
    p = EcoParams(H=30, W=45, p_spont=0.0, p_class=(0.0, 0.5, 0.5, 0.5))
    wall = np.zeros((p.H, p.W), np.uint8)
    wall[0, :] = wall[-1, :] = wall[:, 0] = wall[:, -1] = 1
    res = ((rng.random((p.H, p.W)) < 0.05) & (wall == 0)).astype(np.uint8)
    counts = signal.convolve2d(res.astype(np.int64), _kernel(0, 2), mode="same")
    for t in range(50):
        new = oracle.regrow(p.asdict(), 3, t, res, wall)
        assert np.all(new[res == 1] == 1)            # resources persist
        assert np.all(new[wall == 1] == 0)           # walls never grow
        assert np.all(new[(counts == 0) & (res == 0)] == 0)  # no spontaneous growth
    # every probability zero: the grid never changes
    q = p.replace(p_class=(0.0, 0.0, 0.0, 0.0))
    for t in range(20):
        np.testing.assert_array_equal(oracle.regrow(q.asdict(), 3, t, res, wall), res)
    # spontaneous growth reaches isolated cells at rate p_spont
    q = p.replace(p_class=(0.0, 0.0, 0.0, 0.0), p_spont=0.05)
    empty0 = (counts == 0) & (res == 0) & (wall == 0)
    k = sum(int((oracle.regrow(q.asdict(), 3, t, res, wall) & empty0).sum()) for t in range(100))
    n = int(empty0.sum()) * 100
    assert stats.binomtest(k, n, 0.05).pvalue > 1e-4
    assert math.isfinite(k)
