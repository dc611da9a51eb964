"""Pins of the oracle's whole step: initial state, moves, physiology, births.

Initial state is rebuilt from an independent numpy Philox; energies follow
the float32 sequence computed here with numpy; moves and births are checked
by brute force against their declarative definitions on <=4x4 worlds; a free
run of the 20x40 world is checked against the invariants (one agent per
cell, population bookkeeping, energy bookkeeping, slot assignment).
"""
import itertools
import math

import numpy as np
import pytest

from paper_2302_09334_gb300.params import INT32_MAX, EcoParams, small_20x40
from tests import philox_np

DY = [0, -1, 1, 0, 0]
DX = [0, 0, 0, 1, -1]


def _np_normals(seed, tag, t, ident, n):
    """Normals 0..n-1 of the stream (seed, tag, t, ident), numpy Box-Muller."""
    q = np.arange((n + 3) // 4, dtype=np.uint32)
    r = philox_np.philox(q, t, tag, ident, seed & 0xFFFFFFFF, seed >> 32)
    u = [(x.astype(np.float64) + 0.5) / 2**32 for x in r]
    rad0 = np.sqrt(-2 * np.log(u[0]))
    rad1 = np.sqrt(-2 * np.log(u[2]))
    z = np.stack([rad0 * np.cos(2 * np.pi * u[1]), rad0 * np.sin(2 * np.pi * u[1]),
                  rad1 * np.cos(2 * np.pi * u[3]), rad1 * np.sin(2 * np.pi * u[3])], -1)
    return z.ravel()[:n]


def test_initial_state_reconstruction(oracle):
    p = small_20x40()
    seed = 0
    w = oracle.OracleWorld(p.asdict(), seed)
    H, W = p.H, p.W
    wall = np.zeros((H, W), np.uint8)
    wall[0, :] = wall[-1, :] = wall[:, 0] = wall[:, -1] = 1
    np.testing.assert_array_equal(w.wall, wall)
    u = philox_np.grid_words(seed, H, W, 0, 3)
    res = ((u < math.floor(0.1 * 2**32)) & (wall == 0)).astype(np.uint8)
    np.testing.assert_array_equal(w.res, res)
    key = philox_np.grid_words(seed, H, W, 0, 2).ravel().astype(np.uint64)
    cells = np.arange(H * W, dtype=np.uint64)
    free = wall.ravel() == 0
    order = np.argsort((key[free] << np.uint64(32)) | cells[free], kind="stable")
    chosen = cells[free][order][:p.n_agents0].astype(np.int64)
    np.testing.assert_array_equal(w.y[:64] * W + w.x[:64], chosen)
    assert w.alive[:64].all() and not w.alive[64:].any()
    assert np.all(w.energy[:64] == np.float32(1.0))
    for s in (0, 17, 63):
        z = _np_normals(seed, 4, 0, s, 23333)
        want = (np.float64(np.float32(0.1)) * z).astype(np.float32)
        np.testing.assert_allclose(w.weights[s], want, rtol=0, atol=1e-7 * 0.1)
    assert np.all(w.weights[64:] == 0)


def _empty_world(oracle, H, W, C, **kw):
    base = dict(H=H, W=W, capacity=C, n_agents0=0, border_walls=0, res_init_p=0.0,
                p_class=(0.0, 0.0, 0.0, 0.0), p_spont=0.0, e_decay=0.0,
                t_repr=INT32_MAX)
    base.update(kw)
    p = EcoParams(**base)
    return p, oracle.OracleWorld(p.asdict(), 1)


def _place(w, agents):
    w.alive[:] = 0
    for s, (y, x) in agents.items():
        w.alive[s] = 1
        w.y[s], w.x[s] = y, x
        w.energy[s] = np.float32(1.0)
    w.sync()


def test_never_eating_agent_float32_trajectory(oracle):
    # one agent, no resources: energy falls by 0.01 (float32) per step, the
    # reproduction counter counts steps with energy > 0.5, death at <= 0
    p, w = _empty_world(oracle, 9, 9, 4, e_decay=0.01, t_repr=50)
    _place(w, {0: (4, 4)})
    e = np.float32(1.0)
    ctr = 0
    birth_step = death_step = None
    for k in range(1, 121):
        e = np.float32(e - np.float32(0.01))
        ctr = ctr + 1 if e > np.float32(0.5) else 0
        if birth_step is None and ctr >= 50:
            birth_step = k
        if death_step is None and e <= 0:
            death_step = k
    # float32 rounding: 50 steps stay above 0.5, and 1 - 100*0.01 is not 0
    assert birth_step == 50 and death_step == 101
    for k in range(1, 121):
        w.step(forced=np.zeros(4, np.int32))
        assert w.counters[oracle.C_BIRTHS_LAST] == (1 if k in (50, 100) else 0), k
        if k == birth_step:
            assert w.repr_ctr[0] == 0 and w.alive[1] == 1
        assert w.alive[0] == (1 if k < death_step else 0), k


def test_energy_bookkeeping_with_eating(oracle):
    p, w = _empty_world(oracle, 6, 6, 2, e_decay=0.01, e_gain=0.2, e_max=1.5)
    _place(w, {0: (2, 2)})
    w.res[2, 3] = 1
    w.res[2, 4] = 1
    e = np.float32(1.0)
    for a in (3, 3, 0, 0):
        ate = False
        y, x = w.y[0], w.x[0]
        ny, nx = y + DY[a], x + DX[a]
        if w.res[ny, nx]:
            ate = True
        w.step(forced=np.array([a, 0], np.int32))
        if ate:
            e = np.float32(e + np.float32(0.2))
        e = np.float32(e - np.float32(0.01))
        e = min(e, np.float32(1.5))
        assert w.energy[0] == e and w.ate[0] == ate
    assert w.res.sum() == 0


def _brute_moves(alive, pos, wall, acts, H, W):
    occ = {pos[s] for s in alive}
    claims = {}
    for s in sorted(alive):
        a = acts[s]
        if a == 0:
            continue
        t = (pos[s][0] + DY[a], pos[s][1] + DX[a])
        if not (0 <= t[0] < H and 0 <= t[1] < W) or wall[t] or t in occ:
            continue
        claims.setdefault(t, []).append(s)
    new = dict(pos)
    for t, ss in claims.items():
        new[min(ss)] = t
    return new


@pytest.mark.parametrize("H,W,k", [(3, 3, 3), (4, 4, 4), (2, 4, 3)])
def test_moves_brute_force(oracle, H, W, k):
    rng = np.random.default_rng(H * 10 + W + k)
    for trial in range(4):
        p, w = _empty_world(oracle, H, W, k + 1)
        wall = (rng.random((H, W)) < 0.15).astype(np.uint8)
        free = [(y, x) for y in range(H) for x in range(W) if not wall[y, x]]
        if len(free) < k:
            continue
        cells = [free[i] for i in rng.choice(len(free), k, replace=False)]
        slots = sorted(rng.choice(k + 1, k, replace=False).tolist())
        agents = dict(zip(slots, cells))
        for acts in itertools.product(range(5), repeat=k):
            w.wall[:] = wall
            _place(w, agents)
            forced = np.zeros(k + 1, np.int32)
            forced[slots] = acts
            w.step(forced=forced)
            want = _brute_moves(slots, agents, wall, dict(zip(slots, acts)), H, W)
            got = {s: (int(w.y[s]), int(w.x[s])) for s in slots}
            assert got == want, (agents, acts)
            assert len(set(got.values())) == k
            for s, (y, x) in got.items():
                assert w.slot_map[y, x] == s


def test_wall_kills(oracle):
    p, w = _empty_world(oracle, 4, 4, 3, wall_kills=1)
    w.wall[0, 1] = 1
    _place(w, {0: (1, 1), 1: (3, 3)})
    w.step(forced=np.array([1, 2, 0], np.int32))  # 0 -> wall, 1 -> off the grid
    assert w.alive[0] == 0 and w.alive[1] == 0
    assert w.counters[oracle.C_DEATHS_LAST] == 2 and w.population == 0
    assert np.all(w.slot_map == -1)


def _brute_births(alive, pos, wall, H, W, C):
    occ = {pos[s] for s in alive}
    cand = {}
    for s in sorted(alive):
        for a in (1, 2, 3, 4):
            c = (pos[s][0] + DY[a], pos[s][1] + DX[a])
            if 0 <= c[0] < H and 0 <= c[1] < W and not wall[c] and c not in occ:
                cand[s] = c
                break
    winners = sorted(s for s, c in cand.items() if min(q for q, d in cand.items() if d == c) == s)
    free = [s for s in range(C) if s not in alive]
    return [(par, free[i], cand[par]) for i, par in enumerate(winners) if i < len(free)], \
        max(0, len(winners) - len(free))


@pytest.mark.parametrize("H,W,C", [(3, 3, 4), (4, 4, 6), (4, 4, 3), (1, 4, 4)])
def test_births_brute_force(oracle, H, W, C):
    rng = np.random.default_rng(H * 100 + W * 10 + C)
    for trial in range(40):
        p, w = _empty_world(oracle, H, W, C, t_repr=1, e_repr=0.5)
        wall = (rng.random((H, W)) < 0.2).astype(np.uint8)
        free = [(y, x) for y in range(H) for x in range(W) if not wall[y, x]]
        k = int(rng.integers(1, min(C, len(free)) + 1)) if free else 0
        if k == 0:
            continue
        cells = [free[i] for i in rng.choice(len(free), k, replace=False)]
        slots = sorted(rng.choice(C, k, replace=False).tolist())
        agents = dict(zip(slots, cells))
        w.wall[:] = wall
        _place(w, agents)
        w.step(forced=np.zeros(C, np.int32))
        want, dropped = _brute_births(slots, agents, wall, H, W, C)
        nb = int(w.counters[oracle.C_BIRTHS_LAST])
        got = [(int(w.birth_parent[i]), int(w.birth_child[i]),
                (int(w.y[w.birth_child[i]]), int(w.x[w.birth_child[i]]))) for i in range(nb)]
        assert got == want
        assert int(w.counters[oracle.C_DROPPED_LAST]) == dropped
        for par, child, _ in want:
            assert w.repr_ctr[par] == 0 and w.alive[child] == 1
            assert w.energy[child] == np.float32(p.e0) and w.age[child] == 0
        assert w.population == k + nb
        assert int(w.alive.sum()) == k + nb


def test_mutation_statistics(oracle):
    p, w = _empty_world(oracle, 3, 3, 2, t_repr=1, mut_std=0.02)
    _place(w, {0: (1, 1)})
    w.weights[0] = np.linspace(-1, 1, 23333, dtype=np.float32)
    w.step(forced=np.zeros(2, np.int32))
    assert w.counters[oracle.C_BIRTHS_LAST] == 1
    d = w.weights[1].astype(np.float64) - w.weights[0].astype(np.float64)
    n = d.size
    assert abs(d.mean()) < 4 * 0.02 / math.sqrt(n)
    assert abs(d.std() - 0.02) < 4 * 0.02 * math.sqrt(0.5 / n)
    # the noise is keyed by (step, parent): it is normal j of (TAG_MUT, t=0, parent 0)
    z = _np_normals(1, 5, 0, 0, 23333)
    want = (w.weights[0].astype(np.float64) + np.float64(np.float32(0.02)) * z).astype(np.float32)
    np.testing.assert_allclose(w.weights[1], want, rtol=0, atol=2e-9)


def test_death_rules(oracle):
    # paper-form death: energy at or below e_death for t_death steps, or age
    p, w = _empty_world(oracle, 5, 5, 3, e_decay=0.5, t_death=3, max_age=INT32_MAX)
    _place(w, {0: (2, 2)})
    alive_after = []
    for _ in range(6):
        w.step(forced=np.zeros(3, np.int32))
        alive_after.append(int(w.alive[0]))
    # energy 1.0 -> 0.5 -> 0.0 (low 1) -> -0.5 (2) -> -1.0 (3: dies)
    assert alive_after == [1, 1, 1, 0, 0, 0]
    p, w = _empty_world(oracle, 5, 5, 3, max_age=4)
    _place(w, {0: (2, 2)})
    alive_after = []
    for _ in range(6):
        w.step(forced=np.zeros(3, np.int32))
        alive_after.append(int(w.alive[0]))
    assert alive_after == [1, 1, 1, 1, 0, 0]


def test_free_run_invariants(oracle):
    p = small_20x40()
    w = oracle.OracleWorld(p.asdict(), 0)
    pop = w.population
    births_seen = 0
    agent_steps = 0
    for step in range(300):
        e_before = w.energy.copy()
        alive_before = w.alive.copy()
        agent_steps += int(alive_before.sum())     # agents that act in this step
        w.step()
        c = w.counters
        assert c[oracle.C_AGENT_STEPS] == agent_steps
        assert w.population == pop + c[oracle.C_BIRTHS_LAST] - c[oracle.C_DEATHS_LAST]
        pop = w.population
        births_seen += int(c[oracle.C_BIRTHS_LAST])
        alive = np.flatnonzero(w.alive)
        assert len(alive) == pop
        cells = w.y[alive] * p.W + w.x[alive]
        assert len(np.unique(cells)) == pop                 # one agent per cell
        assert not w.wall.ravel()[cells].any()              # never on a wall
        sm = w.slot_map.ravel()
        assert np.all(sm[cells] == alive) and (sm >= 0).sum() == pop
        children = set(w.birth_child[:c[oracle.C_BIRTHS_LAST]].tolist())
        for s in alive:
            if s in children:
                assert w.energy[s] == np.float32(1.0)
                continue
            assert alive_before[s]
            e = e_before[s]
            if w.ate[s]:
                e = np.float32(e + np.float32(0.2))
            e = np.float32(e - np.float32(0.01))
            assert w.energy[s] == e
        old = np.array([s for s in alive if s not in children], np.int64)
        if len(old):   # every agent that was alive before the step ate its cell
            assert not w.res.ravel()[w.y[old] * p.W + w.x[old]].any()
    assert births_seen > 0 and w.t == 300
