"""Pins of the oracle's lab-environment greediness (App. C): T_r counts the
windows in which a resource was in the agent's field of view, C_r those in
which it ate; G = C_r / T_r.  Hand-counted walks past placed resources for
both controllers' views (7x7 and 15x15), and a free run recounted from the
states around every step."""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams, lab

E = 3


def _corridor(oracle, controller, xs_res, x0=1, width=30):
    p = lab(EcoParams(H=3, W=width, controller=controller, e_decay=0.0), 0.0)
    ow = oracle.OracleWorld(p.asdict(), 1)
    ow.alive[0], ow.y[0], ow.x[0] = 1, 1, x0
    ow.res[:] = 0
    for x in xs_res:
        ow.res[1, x] = 1
    ow.sync()
    return ow


@pytest.mark.parametrize("controller,radius", [(0, 3), (1, 7)])
def test_hand_counted_windows(oracle, controller, radius):
    # one resource at x = 12; the agent walks east from x = 1, one cell per step
    ow = _corridor(oracle, controller, [12])
    seen_steps, ate_step = [], None
    for k in range(16):
        x_before = int(ow.x[0])
        ow.step(np.array([E], np.int32))
        if abs(x_before - 12) <= radius and (ate_step is None):
            seen_steps.append(k)
        if ow.ate[0]:
            ate_step = k
        if (k + 1) % 4 == 0:
            ow.lab_window()
    # observation at x = 1 + k before step k: in view once 12 - (1 + k) <= radius;
    # it eats in step 10 (moving from x = 11 onto x = 12)
    assert ate_step == 10
    first_seen = 12 - radius - 1
    assert seen_steps[0] == first_seen
    windows_seen = {k // 4 for k in range(first_seen, 11)}   # gone once eaten
    assert int(ow.lab_t[0]) == len(windows_seen)
    assert int(ow.lab_c[0]) == 1


def test_nothing_in_view_counts_nothing(oracle):
    ow = _corridor(oracle, 0, [25])
    for k in range(8):
        ow.step(np.array([0], np.int32))          # stays at x = 1
        if (k + 1) % 4 == 0:
            ow.lab_window()
    assert int(ow.lab_t[0]) == 0 and int(ow.lab_c[0]) == 0


def test_free_run_recount(oracle):
    """Several agents, regrowth on, windows of 20: T_r and C_r recounted from
    each step's views and meals; C_r <= T_r (a meal is always in view)."""
    p = EcoParams(H=20, W=40, capacity=128, n_agents0=30, e_decay=0.005, t_repr=40,
                  e_repr=0.8)
    ow = oracle.OracleWorld(p.asdict(), 2)
    seen = np.zeros(p.capacity, np.int64)
    ate = np.zeros(p.capacity, np.int64)
    T = np.zeros(p.capacity, np.int64)
    Cc = np.zeros(p.capacity, np.int64)
    for k in range(120):
        live = np.flatnonzero(ow.alive)
        t = ow.t
        regrown = oracle.regrow(p.asdict(), 2, t, ow.res, ow.wall)
        view = {}
        for s in live:
            obs = oracle.observe(p.asdict(), regrown, ow.wall, ow.slot_map, ow.y[s], ow.x[s],
                                 ow.energy[s])
            view[s] = obs[:49].any()
        ow.step()
        nb = int(ow.counters[5])
        for ch in ow.birth_child[:nb]:
            seen[ch] = ate[ch] = T[ch] = Cc[ch] = 0
        for s in live:
            if s in set(int(v) for v in ow.birth_child[:nb]):
                continue
            seen[s] |= view[s]
            ate[s] |= int(ow.ate[s])
        if (k + 1) % 20 == 0:
            alive = ow.alive.astype(bool)
            T[alive] += seen[alive]
            Cc[alive] += ate[alive]
            seen[:] = 0
            ate[:] = 0
            ow.lab_window()
            np.testing.assert_array_equal(ow.lab_t[alive], T[alive])
            np.testing.assert_array_equal(ow.lab_c[alive], Cc[alive])
            assert np.all(ow.lab_c[alive] <= ow.lab_t[alive])
    assert Cc.sum() > 0
