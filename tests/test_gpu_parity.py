"""Parity of the CUDA step with the CPU oracle (GPU tests).

Every case starts both sides from the same seed (or the same loaded state),
steps them with the oracle's actions forced on the GPU, and compares the
full state after each step under the rules in tests/parity.py.
"""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import INT32_MAX, EcoParams, paper_200x400, small_20x40
from tests import inputs
from tests.parity import compare, run_forced, weights_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eco():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    return world


def _pair(eco, oracle, p, seed):
    gw = eco.World(p, seed)
    ow = oracle.OracleWorld(p.asdict(), seed)
    return gw, ow


def test_initial_state_matches(eco, oracle):
    p = small_20x40()
    gw, ow = _pair(eco, oracle, p, 0)
    gs = gw.read_state(weights=(0, p.capacity))
    compare(gs, ow, "init")
    weights_close(gs["weights"][:p.n_agents0], ow.weights[:p.n_agents0], p.w_init_std, "init weights")


def test_small_world_500_steps_forced(eco, oracle):
    p = small_20x40()
    gw, ow = _pair(eco, oracle, p, 0)
    st = run_forced(gw, ow, 500, "20x40", p.mut_std)
    assert st["births"] > 0
    assert ow.counters[3] > 0  # deaths happened too


def test_small_world_wide_weights_forced(eco, oracle):
    """Initial weights N(0, 0.5^2): pre-activations of tens, saturated gates,
    logits with large cancellations; the RNN tolerance is the same per-element
    bound on the oracle's error magnitudes."""
    p = small_20x40().replace(w_init_std=0.5)
    gw, ow = _pair(eco, oracle, p, 1)
    st = run_forced(gw, ow, 300, "20x40 std 0.5", p.mut_std)
    print("std 0.5:", st)
    assert st["births"] > 0 and st["budget"] <= 1.0
    assert st["flagged"] <= 5


EDGE_CASES = {
    "ragged_9x33": EcoParams(H=9, W=33, capacity=40, n_agents0=20),
    "paper_forms_24x100": EcoParams(H=24, W=100, capacity=120, n_agents0=60, nbr_shape=1,
                                    nbr_radius=1, class_edges=(1, 2, 5),
                                    p_class=(0.0, 0.05, 0.0, 0.0), lat_mode=1,
                                    p_spont=5e-4, wall_kills=1, t_death=3, max_age=80,
                                    e_max=1.2, e_gain=1.0, t_repr=10, e_decay=0.025),
    "no_agents": EcoParams(H=16, W=70, capacity=8, n_agents0=0, p_class=(0.0, 0.05, 0.1, 0.2)),
    "full_capacity": EcoParams(H=12, W=40, capacity=30, n_agents0=30, t_repr=5),
    "tiny_3x3": EcoParams(H=3, W=3, capacity=4, n_agents0=1, t_repr=3),
    "radius3_open": EcoParams(H=17, W=65, capacity=64, n_agents0=40, border_walls=0,
                              nbr_radius=3, class_edges=(1, 4, 9), e_decay=0.02),
    "word_multiple_8x64": EcoParams(H=8, W=64, capacity=64, n_agents0=32, t_repr=7),
    # capacity above 16384: the slot phases run as five multi-CTA kernels
    "split_path_cap20000": EcoParams(H=40, W=80, capacity=20000, n_agents0=400, t_repr=20),
}


@pytest.mark.parametrize("name", list(EDGE_CASES))
def test_edge_cases_forced(eco, oracle, name):
    p = EDGE_CASES[name]
    gw, ow = _pair(eco, oracle, p, 11)
    compare(gw.read_state(), ow, f"{name} init")
    run_forced(gw, ow, 120, name, p.mut_std)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_from_identical_random_state(eco, oracle, seed):
    p = EcoParams(H=30, W=75, capacity=300, n_agents0=0, t_repr=3, e_decay=0.01)
    state = inputs.random_state(p, seed, n_agents=180, t=1000 + seed)
    gw, ow = _pair(eco, oracle, p, 5)
    inputs.load_into_oracle(ow, state)
    gw.load_state(state)
    compare(gw.read_state(), ow, "loaded")
    st = run_forced(gw, ow, 25, f"random state {seed}", p.mut_std)
    assert st["births"] > 0


def test_paper_scale_world_forced(eco, oracle):
    p = paper_200x400()
    gw, ow = _pair(eco, oracle, p, 0)
    gs = gw.read_state(weights=(0, 64))
    compare(gs, ow, "200x400 init")
    weights_close(gs["weights"], ow.weights[:64], p.w_init_std, "200x400 init weights")
    run_forced(gw, ow, 60, "200x400", p.mut_std, compare_every=10)


def test_load_state_pinned_equals_pageable(eco):
    """A state loaded from page-locked host memory (weights read by the
    device through its address) equals the same state loaded from pageable
    memory (2-D copy and in-place permutation), for both controllers and a
    weight count whose floats are not a multiple of four."""
    import torch
    for p in (EcoParams(H=30, W=60, capacity=300, n_agents0=120),
              EcoParams(H=30, W=60, capacity=300, n_agents0=120, controller=1)):
        src = eco.World(p, 3)
        src.step(30)
        n = 117                                    # 117 * 23333 and 117 * 2445 are odd
        st = src.read_state(weights=(0, n))
        pinned = {}
        for k, v in st.items():
            t = torch.empty(v.shape, dtype=torch.from_numpy(v[:0].copy()).dtype, pin_memory=True)
            pinned[k] = t.numpy()
            pinned[k][...] = v
        a, b = eco.World(p, 9), eco.World(p, 9)
        a.load_state(pinned)
        b.load_state({k: np.array(v) for k, v in st.items()})
        ra, rb = a.read_state(weights=(0, n)), b.read_state(weights=(0, n))
        for k in ra:
            np.testing.assert_array_equal(ra[k], rb[k], err_msg=k)
        np.testing.assert_array_equal(ra["weights"], st["weights"])
        a.step(10)
        b.step(10)
        ra, rb = a.read_state(weights=(0, p.capacity)), b.read_state(weights=(0, p.capacity))
        live = ra["alive"].astype(bool)
        np.testing.assert_array_equal(ra["weights"][live], rb["weights"][live])
        np.testing.assert_array_equal(ra["h"], rb["h"])
        for w in (src, a, b):
            w.close()


def test_free_run_is_deterministic(eco):
    p = small_20x40()
    a = eco.World(p, 3)
    b = eco.World(p, 3)
    a.step(200)
    b.step(57)
    b.step(143)
    sa, sb = a.read_state(), b.read_state()
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)


def test_batch_equals_alone(eco):
    import torch
    ps = [small_20x40(), EcoParams(H=33, W=90, capacity=200, n_agents0=100),
          EcoParams(H=50, W=100, capacity=400, n_agents0=150, lat_bottom=0.6)]
    stream = torch.cuda.Stream()
    alone = [eco.World(p, 10 + i) for i, p in enumerate(ps)]
    mixed = [eco.World(p, 10 + i, stream=stream) for i, p in enumerate(ps)]
    for w in alone:
        w.step(150)
    batch = eco.Batch(mixed)
    batch.step(150)
    batch.sync()
    for wa, wb in zip(alone, mixed):
        sa, sb = wa.read_state(), wb.read_state()
        for k in sa:
            np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)


def test_load_state_keeping_counters_and_a_weight_range(eco):
    """load_state with set_counters=False keeps the device's counters (the
    step counter, read back, decides which buffer of the plane and h pairs
    is current), and a weight range starting past slot 0 replaces exactly
    those rows: the world then steps as the one the state was read from
    (same seed, so the same random streams)."""
    p = EcoParams(H=30, W=60, capacity=400, n_agents0=150, t_repr=20, e_repr=0.4)
    src = eco.World(p, 21)
    src.step(37)                                  # odd step counter
    st = src.read_state(weights=(0, p.capacity))
    # the same seed (the random streams are keyed by it, not by the state),
    # another history: the initial state of seed 22, then as many steps
    other = eco.World(p, 22)
    dst = eco.World(p, 21)
    dst.load_state(other.read_state(weights=(0, p.capacity)))
    other.close()
    dst.step(37)                                  # same step counter
    c_dst = dst.read_state(fields=())["counters"]
    assert c_dst[0] == st["counters"][0] and c_dst[2] != st["counters"][2]
    dst.load_state({k: v for k, v in st.items() if k != "weights"}, set_counters=False)
    c_after = dst.read_state(fields=())["counters"]
    np.testing.assert_array_equal(c_after[[0, 2, 3, 4]], c_dst[[0, 2, 3, 4]])  # t, cumulative
    assert c_after[1] == st["counters"][1]        # population: the loaded alive flags
    # weights in two ranges, the second starting past slot 0
    lo = 137
    dst.load_state({"weights": st["weights"][:lo]}, set_counters=False, weights_first=0)
    dst.load_state({"weights": st["weights"][lo:]}, set_counters=False, weights_first=lo)
    mid = dst.read_state(weights=(0, p.capacity))
    for k in ("alive", "y", "x", "energy", "h", "c", "res", "wall", "weights"):
        np.testing.assert_array_equal(mid[k], st[k], err_msg=k)
    src.step(25)
    dst.step(25)
    a, b = src.read_state(weights=(0, p.capacity)), dst.read_state(weights=(0, p.capacity))
    assert a["counters"][2] > st["counters"][2]   # births in the 25 steps
    for k in a:
        if k == "counters":
            np.testing.assert_array_equal(a[k][[0, 1, 5, 6, 7]], b[k][[0, 1, 5, 6, 7]])
        else:
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    src.close()
    dst.close()


def test_load_rejects_inconsistent_state(eco):
    from paper_2302_09334_gb300._lib import EcoError, ECO_ESTATE
    p = EcoParams(H=8, W=8, capacity=4, n_agents0=2)
    w = eco.World(p, 0)
    st = w.read_state()
    st["alive"][:] = [1, 1, 0, 0]
    st["y"][:2] = 3
    st["x"][:2] = 4
    with pytest.raises(EcoError) as e:
        w.load_state(st)
    assert e.value.code == ECO_ESTATE
    st["y"][1] = 0  # on the border wall
    with pytest.raises(EcoError):
        w.load_state(st)
    st["y"][1] = 2
    w.load_state(st)  # consistent again
    w.step(3)
    w.sync()


def test_held_population_stays_constant(eco):
    p = small_20x40().replace(e_decay=0.0, t_repr=INT32_MAX)
    w = eco.World(p, 4)
    w.step(100)
    c = w.counters()
    assert c[1] == p.n_agents0 and c[2] == 0 and c[3] == 0


def test_checkpoint_resume_is_exact(eco):
    """n steps straight == k steps, save, load into a fresh world of the same
    seed, n - k steps (every field, every weight, bit for bit)."""
    p = small_20x40().replace(capacity=400, max_age=150)
    a = eco.World(p, seed=31)
    a.step(300)
    b = eco.World(p, seed=31)
    b.step(120)
    saved = b.read_state(weights=(0, p.capacity))
    b.close()
    c = eco.World(p, seed=31)
    c.step(7)                     # whatever it held before is replaced
    c.load_state(saved)
    c.step(180)
    sa = a.read_state(weights=(0, p.capacity))
    sc = c.read_state(weights=(0, p.capacity))
    live = sa["alive"].astype(bool)
    for k in sa:
        if k in ("h", "c", "logits", "weights", "action", "prev_action", "ate", "y", "x",
                 "energy", "repr_ctr", "low_ctr", "age"):
            np.testing.assert_array_equal(sa[k][live], sc[k][live], err_msg=k)
        else:
            np.testing.assert_array_equal(sa[k], sc[k], err_msg=k)
    assert int(sa["counters"][0]) == 300 and sa["counters"][2] > 0
    a.close()
    c.close()
