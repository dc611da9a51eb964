"""The step's result does not depend on the order in which slots are
visited (the CUDA kernels visit them in no fixed order): the oracle's
per-slot loops run in ascending order, or in a permutation installed by its
test hook, and every field must come out the same, bit for bit.  The
ranking of births (the k-th successful parent in ascending slot order gets
the k-th free slot) is an order the method defines and is not permuted.

Workloads: the 20x40 configuration free-running through its first birth
bursts, and a crowded 8x8 world with random forced moves (most targets are
contested), quick reproduction, walls that kill and a capacity that drops
births.
"""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams, small_20x40

FIELDS = ("res", "slot_map", "alive", "y", "x", "energy", "repr_ctr", "low_ctr", "age",
          "h", "c", "action", "logits", "ate", "weights", "counters", "birth_parent",
          "birth_child", "move_action", "prev_action", "lab_flags")


def _snapshot(w, n_births):
    snap = {f: getattr(w, f).copy() for f in FIELDS}
    # birth lists: only the entries of this step are defined
    snap["birth_parent"] = snap["birth_parent"][:n_births]
    snap["birth_child"] = snap["birth_child"][:n_births]
    return snap


def _run_pair(oracle, p, seed, steps, forced_fn=None, perm_seed=1):
    """Step an ascending world and a permuted one side by side; compare all
    fields after every step."""
    a = oracle.OracleWorld(p.asdict(), seed)
    b = oracle.OracleWorld(p.asdict(), seed)
    rng = np.random.default_rng(perm_seed)
    C = p.capacity
    births = 0
    for t in range(steps):
        b.set_order(rng.permutation(C))           # a new order every step
        forced = forced_fn(t) if forced_fn else None
        a.step(forced)
        b.step(forced)
        nb = int(a.counters[5])
        births += nb
        sa, sb = _snapshot(a, nb), _snapshot(b, nb)
        for f in FIELDS:
            np.testing.assert_array_equal(sa[f], sb[f], err_msg=f"step {t}: {f}")
    return a, b, births


def test_free_run_independent_of_slot_order(oracle):
    p = small_20x40()
    a, b, births = _run_pair(oracle, p, seed=3, steps=120)
    assert births > 0 and int(a.counters[3]) >= 0
    a.close()
    b.close()


def test_contested_moves_and_births_independent_of_slot_order(oracle):
    p = EcoParams(H=8, W=8, capacity=40, n_agents0=36, border_walls=0, res_init_p=0.5,
                  t_repr=3, e_repr=0.5, e_decay=0.01, wall_kills=1, max_age=60)
    rng = np.random.default_rng(11)
    actions = rng.integers(0, 5, size=(80, p.capacity)).astype(np.int32)
    a, b, births = _run_pair(oracle, p, seed=5, steps=80, forced_fn=lambda t: actions[t])
    assert births > 0                              # births happened
    assert int(a.counters[4]) > 0                  # and some were dropped (capacity 40)
    assert int(a.counters[3]) > 0                  # deaths (walls kill off-grid moves)
    a.close()
    b.close()


def test_paper_controller_independent_of_slot_order(oracle):
    # the paper's controller samples its actions from per-(slot, step) draws
    p = EcoParams(H=20, W=40, capacity=120, n_agents0=60, res_init_p=0.2, t_repr=6,
                  e_repr=0.5, e_decay=0.02, controller=1, max_age=80)
    a, b, births = _run_pair(oracle, p, seed=9, steps=40)
    assert births > 0
    a.close()
    b.close()


def test_set_order_rejects_non_permutations(oracle):
    p = small_20x40()
    w = oracle.OracleWorld(p.asdict(), 0)
    with pytest.raises(ValueError):
        w.set_order(np.zeros(p.capacity, np.int32))          # repeats
    with pytest.raises(ValueError):
        w.set_order(np.arange(1, p.capacity + 1, dtype=np.int32))   # out of range
    w.set_order(np.arange(p.capacity)[::-1].copy())
    w.set_order(None)
    w.close()
