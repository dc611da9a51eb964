"""Full-size parity: the 1000x2000 world (20,000 agents, capacity 131,072,
the split slot kernels and their four-kernel compaction), against the
oracle:

* initial walls, resources and agent placement over the whole grid
  (or_initial_layout), initial weights of sampled agents (or_fill_normals);
* eight steps with the oracle's actions forced, compared with the oracle
  world after every step (grid, slot map, positions, energies, counters,
  h, c, logits, actions, children's weights): a churn variant (initial
  energy 0.045, reproduction after 3 steps above 0) has two waves of about
  20,000 and 26,000 births and one of about 14,000 deaths, so births, slot
  assignment from the free list, the compaction and the mutation all run at
  this size;
* one free step whose regrowth, sampled observations + LSTM steps and
  energies are recomputed piece by piece (an extra check).
"""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import large_1000x2000
from tests.parity import RNN_TOL, compare, rnn_close, run_forced, small_margin, weights_close

pytestmark = pytest.mark.gpu

DY = np.array([0, -1, 1, 0, 0])
DX = np.array([0, 0, 0, 1, -1])


@pytest.fixture(scope="module")
def large():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    p = large_1000x2000()
    gw = world.World(p, seed=0)
    yield p, gw
    gw.close()


def test_large_initial_state(large, oracle):
    p, gw = large
    st = gw.read_state(fields=("res", "wall", "alive", "y", "x", "energy", "slot_map"))
    res, wall, cells = oracle.initial_layout(p.asdict(), 0)
    np.testing.assert_array_equal(st["wall"], wall)
    np.testing.assert_array_equal(st["res"], res)
    n0 = p.n_agents0
    assert st["alive"][:n0].all() and not st["alive"][n0:].any()
    np.testing.assert_array_equal(st["y"][:n0] * p.W + st["x"][:n0], cells)
    assert np.all(st["energy"][:n0] == np.float32(p.e0))
    assert (st["slot_map"] >= 0).sum() == n0
    for s in (0, 1, 777, n0 // 2, n0 - 1):
        g = gw.read_state(fields=(), weights=(s, 1))["weights"][0]
        want = oracle.fill_normals(0, oracle.TAG_INIT_W, 0, s, p.w_init_std)
        weights_close(g, want, p.w_init_std, f"initial weights of slot {s}")


def test_large_one_step(large, oracle):
    p, gw = large
    H, W = p.H, p.W
    before = gw.read_state()
    t = int(before["counters"][0])
    gw.step(1)
    after = gw.read_state()
    live0 = before["alive"].astype(bool)
    reborn = live0 & after["alive"].astype(bool) & (after["age"] == 0)
    known = live0 & ~reborn

    # regrowth over the whole grid; the only other change is eating
    regrown = oracle.regrow(p.asdict(), 0, t, before["res"], before["wall"])
    assert not (after["res"] & ~regrown).any()        # nothing appears but regrowth
    eaten = np.argwhere(regrown & ~after["res"])
    final = set((after["y"][known] * W + after["x"][known]).tolist())
    unexplained = sum(1 for (y, x) in eaten if y * W + x not in final)
    assert unexplained <= int(reborn.sum())

    # observation + LSTM of sampled agents from the state before the step
    rng = np.random.default_rng(0)
    sample = rng.choice(np.flatnonzero(known), 192, replace=False)
    flagged = 0
    for s in sample:
        obs = oracle.observe(p.asdict(), regrown, before["wall"], before["slot_map"],
                             before["y"][s], before["x"][s], before["energy"][s])
        w = gw.read_state(fields=(), weights=(int(s), 1))["weights"][0]
        a, h2, c2, lg = oracle.lstm_step(w, obs, before["h"][s], before["c"][s])
        Eh, Ec, El = oracle.lstm_mag(w, obs, before["h"][s], before["c"][s])
        rnn_close(after["h"][s], h2, Eh, f"h of slot {s}")
        rnn_close(after["c"][s], c2, Ec, f"c of slot {s}")
        rnn_close(after["logits"][s], lg, El, f"logits of slot {s}")
        if after["action"][s] != a:
            assert small_margin(lg[None], El[None])[0], f"action of slot {s}"
            flagged += 1
    assert flagged <= 2

    # the move rule over every agent, with the actions the GPU took
    act = np.where(live0, after["action"], 0)
    ty = before["y"] + DY[act]
    tx = before["x"] + DX[act]
    inb = (ty >= 0) & (ty < H) & (tx >= 0) & (tx < W)
    tcell = np.where(inb, ty * W + tx, 0)
    valid = live0 & (act > 0) & inb
    valid &= before["wall"].ravel()[tcell] == 0
    valid &= before["slot_map"].ravel()[tcell] == -1
    order = np.argsort(np.where(valid, tcell, -1) * (1 << 20) + np.arange(len(act)), kind="stable")
    winner = np.zeros(len(act), bool)
    seen = set()
    for s in order:
        if valid[s] and tcell[s] not in seen:
            seen.add(tcell[s])
            winner[s] = True
    exp_y = np.where(winner, ty, before["y"])
    exp_x = np.where(winner, tx, before["x"])
    np.testing.assert_array_equal(after["y"][known], exp_y[known])
    np.testing.assert_array_equal(after["x"][known], exp_x[known])

    # energy: gain if the final cell had a resource after regrowth, then decay
    cell = exp_y * W + exp_x
    ate = regrown.ravel()[cell].astype(bool)
    e = before["energy"].copy()
    e = np.where(ate, (e + np.float32(p.e_gain)).astype(np.float32), e)
    e = (e - np.float32(p.e_decay)).astype(np.float32)
    surv = known & after["alive"].astype(bool)
    np.testing.assert_array_equal(after["energy"][surv].view(np.uint32), e[surv].view(np.uint32))
    died = live0 & ~after["alive"].astype(bool)
    assert np.all(e[died] <= np.float32(p.e_death))

    # bookkeeping and one agent per cell
    c = after["counters"]
    assert c[1] == before["counters"][1] + c[5] - c[6]
    alive = np.flatnonzero(after["alive"])
    assert len(alive) == c[1]
    sm = after["slot_map"].ravel()
    np.testing.assert_array_equal(sm[after["y"][alive] * W + after["x"][alive]], alive)
    assert (sm >= 0).sum() == len(alive)
    assert RNN_TOL > 0


def test_large_forced_churn_equals_oracle(oracle):
    """Eight steps of the full-size world under heavy churn, the GPU moving
    with the oracle's actions, compared with the oracle after every step."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    p = large_1000x2000().replace(e0=0.045, e_repr=0.0, t_repr=3)
    gw = world.World(p, seed=0)
    ow = oracle.OracleWorld(p.asdict(), 0)
    try:
        compare(gw.read_state(), ow, "churn init")
        st = run_forced(gw, ow, 8, "1000x2000 churn", p.mut_std)
        c = ow.counters
        print("1000x2000 churn:", dict(births=int(c[2]), deaths=int(c[3]), pop=int(c[1]),
                                       flagged=st["flagged"], budget=st["budget"], rel=st["rel"]))
        assert c[2] > 40000 and c[3] > 10000, "two birth waves and a death wave expected"
        assert st["flagged"] <= 4
    finally:
        gw.close()
        ow.close()
