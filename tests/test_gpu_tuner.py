"""Launch configurations and the tuner: every configuration gives the same
state bit for bit, the tuner's steps are ordinary steps, and invalid
configurations are refused."""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eco():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    return world


def _state(w, p):
    st = w.read_state(weights=(0, p.capacity))
    live = st["alive"].astype(bool)
    st["weights"] = st["weights"][live]
    for f in ("h", "c", "logits", "y", "x", "energy", "repr_ctr", "low_ctr", "age", "action"):
        st[f] = st[f][live]
    return st


def _equal(a, b, where):
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=f"{where}: {k}")


P = EcoParams(H=30, W=60, capacity=600, n_agents0=150, t_repr=25, e_repr=0.4, max_age=140)


def test_every_config_gives_the_same_state(eco):
    configs = [(1, 4, 16), (0, 4, 16), (1, 1, 1), (0, 8, 64), (1, 32, 5)]
    worlds = []
    for fused, sp, k in configs:
        w = eco.World(P, seed=17)
        w.set_config(fused=fused, spawn_ctas_per_sm=sp, steps_per_graph=k)
        assert w.get_config() == {"fused": fused, "spawn_ctas_per_sm": sp, "steps_per_graph": k}
        worlds.append(w)
    for n in (37, 150, 113):
        for w in worlds:
            w.step(n)
        ref = _state(worlds[0], P)
        assert ref["counters"][2] > 0          # births happened
        for (cfg, w) in zip(configs[1:], worlds[1:]):
            _equal(ref, _state(w, P), f"config {cfg} after {int(ref['counters'][0])} steps")
    for w in worlds:
        w.close()


# 70 rows: 9 tiles of 8 rows, stacked 2, 4 and 8 per CTA leave ragged columns
PS = EcoParams(H=70, W=200, capacity=1200, n_agents0=300, t_repr=25, e_repr=0.4, max_age=140)


def test_every_shape_gives_the_same_state(eco):
    shapes = [(1, 1), (2, 2), (4, 1), (8, 2), (0, 2)]
    worlds = []
    for rk, lc in shapes:
        w = eco.World(PS, seed=23)
        w.set_shape(regrow_rows_per_cta=rk, lstm_ctas_per_sm=lc)
        got = w.get_shape()
        assert got["lstm_ctas_per_sm"] == lc
        assert got["regrow_rows_per_cta"] == (rk if rk else got["regrow_rows_per_cta"])
        assert got["regrow_rows_per_cta"] in (1, 2, 4, 8)
        worlds.append(w)
    for n in (30, 90):
        for w in worlds:
            w.step(n)
        ref = _state(worlds[0], PS)
        assert ref["counters"][2] > 0          # births happened
        for (sh, w) in zip(shapes[1:], worlds[1:]):
            _equal(ref, _state(w, PS), f"shape {sh} after {int(ref['counters'][0])} steps")
    # a shape changed between steps continues the same run
    worlds[0].set_shape(regrow_rows_per_cta=8, lstm_ctas_per_sm=2)
    worlds[1].set_shape(regrow_rows_per_cta=1, lstm_ctas_per_sm=1)
    for w in worlds[:2]:
        w.step(20)
    _equal(_state(worlds[0], PS), _state(worlds[1], PS), "shapes swapped")
    for w in worlds:
        w.close()


def test_world_autotune_steps_are_plain_steps(eco):
    a, b = eco.World(P, seed=5), eco.World(P, seed=5)
    r = a.autotune(trial_steps=4)
    assert r["steps_taken"] > 0 and r["ms_per_step_best"] > 0
    cfg = a.get_config()
    assert cfg == {k: r[k] for k in cfg}
    shape = a.get_shape()
    assert shape == {k: r[k] for k in shape}
    b.step(r["steps_taken"])
    _equal(_state(a, P), _state(b, P), "after tuning")
    a.step(40)
    b.step(40)
    _equal(_state(a, P), _state(b, P), "40 steps after tuning")
    a.close()
    b.close()


def test_batch_autotune_equals_alone(eco):
    specs = [(EcoParams(H=20, W=40, n_agents0=60, capacity=240), 1),
             (EcoParams(H=40, W=80, n_agents0=300, capacity=1200), 2),
             (EcoParams(H=12, W=70, n_agents0=40, capacity=160), 3)]
    worlds = [eco.World(p, s) for p, s in specs]
    batch = eco.Batch(worlds)
    r = batch.autotune(trial_steps=2)
    batch.step(25)
    batch.sync()
    for (p, s), w in zip(specs, worlds):
        alone = eco.World(p, s)
        alone.step(r["steps_taken"] + 25)
        _equal(_state(w, p), _state(alone, p), f"world {s}")
        alone.close()
    batch.close()
    for w in worlds:
        w.close()


def test_invalid_configs_refused(eco):
    from paper_2302_09334_gb300._lib import ECO_EINVAL, EcoError
    big = eco.World(EcoParams(H=200, W=200, capacity=20000, n_agents0=100), seed=0)
    assert big.get_config()["fused"] == 0
    for kw in ({"fused": 1}, {"spawn_ctas_per_sm": 0}, {"steps_per_graph": 0},
               {"spawn_ctas_per_sm": 33}):
        with pytest.raises(EcoError) as e:
            big.set_config(**kw)
        assert e.value.code == ECO_EINVAL
    for kw in ({"regrow_rows_per_cta": 3}, {"regrow_rows_per_cta": 16},
               {"lstm_ctas_per_sm": 0}, {"lstm_ctas_per_sm": 3}):
        with pytest.raises(EcoError) as e:
            big.set_shape(**kw)
        assert e.value.code == ECO_EINVAL
    r = big.autotune(trial_steps=1)          # the fused candidate is skipped
    assert r["fused"] == 0
    big.close()
