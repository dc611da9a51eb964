"""Pins of the oracle's analysis metrics (App. C): population, amount of
resources, life expectancy (ages at death over a window) and the 17-bin
histogram of Manhattan displacement over a window.  Each expected value is
counted by hand from a scripted walk or lifetime, or is a second
formulation of the same definition (ages instead of agent identities)."""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams

STAY, N, S, E, W = 0, 1, 2, 3, 4
QUIET = dict(p_class=(0.0, 0.0, 0.0, 0.0), p_spont=0.0, res_init_p=0.0, e_decay=0.0,
             t_repr=2**31 - 1)


def _world(oracle, seed=0, **kw):
    p = EcoParams(**{**dict(H=4, W=12, capacity=8, n_agents0=3), **QUIET, **kw})
    return oracle.OracleWorld(p.asdict(), seed)


def _place(ow, cells):
    ow.alive[:] = 0
    for s, (y, x) in enumerate(cells):
        ow.alive[s], ow.y[s], ow.x[s], ow.age[s] = 1, y, x, 0
    ow.sync()


def test_hand_counted_walks(oracle):
    ow = _world(oracle)
    # interior of the 4x12 world: rows 1-2, columns 1-10
    _place(ow, [(1, 2), (2, 9), (1, 10)])
    a = ow.analysis()
    assert a["window"] == 0 and a["movers"] == 3 and a["move_bins"][0] == 3
    script = [E] * 5 + [W] * 2 + [STAY] * 3                     # slot 0: 2 -> 7 -> 5
    for k in range(10):
        ow.step(np.array([script[k], W, STAY] + [0] * 5, np.int32))
    assert (ow.x[0], ow.x[1], ow.x[2]) == (5, 1, 10)          # slot 1 stops at the wall
    a = ow.analysis()
    assert a["t"] == 10 and a["window"] == 10 and a["population"] == 3
    assert a["movers"] == 3
    want = np.zeros(17, np.int64)
    want[0] += 1          # slot 2: d = 0
    want[4] += 1          # slot 0: d = 3, 3*17 // 11 = 4
    want[12] += 1         # slot 1: d = 8, 8*17 // 11 = 12
    np.testing.assert_array_equal(a["move_bins"], want)
    assert a["deaths"] == 0 and a["death_age_sum"] == 0


def test_fifty_step_window_bins_are_thirds(oracle):
    """With the paper's 50-step window the 51 distances fall in bins of 3."""
    ow = _world(oracle, H=5, W=60, capacity=4)
    _place(ow, [(1, 1), (2, 1), (3, 1)])
    # slot s walks east for 50, 48, 47 steps, then stays
    walk = (50, 48, 47)
    for k in range(50):
        ow.step(np.array([E if k < walk[s] else STAY for s in range(3)] + [0], np.int32))
    a = ow.analysis()
    assert a["window"] == 50 and a["movers"] == 3
    want = np.zeros(17, np.int64)
    want[16] = 2          # 50 // 3 = 16, 48 // 3 = 16
    want[15] = 1          # 47 // 3 = 15
    np.testing.assert_array_equal(a["move_bins"], want)


def test_life_expectancy_closed_form(oracle):
    """No decay and no births: every agent dies of age in step max_age + 1,
    at age max_age + 1."""
    ow = _world(oracle, H=10, W=10, capacity=16, n_agents0=9, max_age=10)
    for _ in range(12):
        ow.step()
    a = ow.analysis()
    assert a["deaths"] == 9 and a["death_age_sum"] == 9 * 11
    assert a["population"] == 0 and a["movers"] == 0 and a["window"] == 12
    b = ow.analysis()     # the next window starts empty
    assert b["window"] == 0 and b["deaths"] == 0 and b["death_age_sum"] == 0


def test_resources_without_regrowth_or_agents(oracle):
    p = EcoParams(**{**dict(H=30, W=50, capacity=4, n_agents0=0), **QUIET, "res_init_p": 0.3})
    res, wall, _ = oracle.initial_layout(p.asdict(), 11)
    ow = oracle.OracleWorld(p.asdict(), 11)
    for _ in range(3):
        ow.step()
    a = ow.analysis()
    assert a["resources"] == int(res.sum()) > 0 and a["population"] == 0


@pytest.mark.parametrize("windows", [(50, 50, 50), (37, 13, 1, 0, 50)])
def test_free_run_against_age_formulation(oracle, windows):
    """Movers are the agents alive over the whole window: by age, the living
    agents with age >= L.  Deaths and their ages are recounted from the
    states before and after every step."""
    p = EcoParams(H=20, W=40, capacity=256, n_agents0=64, e_decay=0.02, t_repr=30,
                  e_repr=0.5, max_age=90)
    ow = oracle.OracleWorld(p.asdict(), 5)
    saw_births = saw_deaths = False
    for L in windows:
        start_cells = np.where(ow.alive.astype(bool), ow.y * p.W + ow.x, -1)
        deaths = age_sum = 0
        for _ in range(L):
            alive0, age0 = ow.alive.astype(bool).copy(), ow.age.copy()
            ow.step()
            alive1 = ow.alive.astype(bool)
            died = alive0 & (~alive1 | (ow.age == 0))    # a freed slot may be reborn
            deaths += int(died.sum())
            age_sum += int((age0[died] + 1).sum())
            saw_births |= int(ow.counters[5]) > 0
        a = ow.analysis()
        assert a["window"] == L
        assert a["deaths"] == deaths and a["death_age_sum"] == age_sum
        saw_deaths |= deaths > 0
        alive = ow.alive.astype(bool)
        movers = alive & (ow.age >= L)
        assert a["movers"] == int(movers.sum()) == int(a["move_bins"].sum())
        assert a["population"] == int(alive.sum()) == ow.population
        assert a["resources"] == int(ow.res.sum())
        y0, x0 = start_cells // p.W, start_cells % p.W
        d = np.abs(ow.y - y0) + np.abs(ow.x - x0)
        assert np.all(d[movers] <= L)
        hist = np.bincount(d[movers] * 17 // (L + 1), minlength=17)
        np.testing.assert_array_equal(a["move_bins"], hist)
    assert saw_births and saw_deaths


def test_sync_rejects_negative_age(oracle):
    ow = _world(oracle)
    ow.age[0] = -1
    with pytest.raises(ValueError):
        ow.sync()
