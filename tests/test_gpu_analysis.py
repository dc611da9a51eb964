"""Analysis metrics of App. C on the GPU (eco_world_analysis_async):
* equal to the oracle's record, integer for integer, on forced runs whose
  windows see births, deaths of energy and age, and wall kills;
* at 200x400 and 1000x2000 (free-running), equal to the same metrics
  recounted on the host from the states at the window ends;
* a batched world's record equals its alone run's; load_state starts a
  window."""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams, large_1000x2000, paper_200x400
from tests.parity import run_forced

pytestmark = pytest.mark.gpu

WINDOWS = (50, 50, 37, 13, 1, 0, 50, 50, 50, 50)


@pytest.fixture(scope="module")
def eco():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    return world


def _same(ga, oa, where):
    assert {k: v for k, v in ga.items() if k != "move_bins"} == \
        {k: v for k, v in oa.items() if k != "move_bins"}, where
    np.testing.assert_array_equal(ga["move_bins"], oa["move_bins"], err_msg=where)


CASES = {
    "small": EcoParams(max_age=120),
    "wall_kills": EcoParams(H=16, W=48, capacity=300, n_agents0=80, wall_kills=1,
                            t_repr=20, e_repr=0.3),
    "ragged_multi_word": EcoParams(H=24, W=71, capacity=512, n_agents0=200, t_repr=25,
                                   e_repr=0.4, max_age=150),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_analysis_equals_oracle(eco, oracle, name):
    p = CASES[name]
    gw = eco.World(p, seed=21)
    ow = oracle.OracleWorld(p.asdict(), 21)
    deaths = births = 0
    try:
        for i, L in enumerate(WINDOWS):
            if L:
                st = run_forced(gw, ow, L, f"{name} window {i}", p.mut_std, compare_every=L)
                births += st["births"]
            ga, oa = gw.analysis(), ow.analysis()
            _same(ga, oa, f"{name} window {i} (L={L})")
            deaths += oa["deaths"]
            assert oa["window"] == L and oa["movers"] == int(oa["move_bins"].sum())
        assert deaths > 0 and births > 0
    finally:
        gw.close()
        ow.close()


@pytest.mark.parametrize("preset,windows", [(paper_200x400, (50, 50, 50)),
                                             (large_1000x2000, (6, 4))])
def test_analysis_recounted_on_host(eco, preset, windows):
    p = preset()
    gw = eco.World(p, seed=3)
    try:
        gw.step(20)
        gw.analysis()                                   # window starts here
        start = gw.read_state(fields=("alive", "y", "x"))
        for L in windows:
            gw.step(L)
            a = gw.analysis()
            st = gw.read_state(fields=("alive", "y", "x", "age", "res"))
            alive = st["alive"].astype(bool)
            movers = alive & (st["age"] >= L)
            assert (start["alive"].astype(bool) | ~movers).all()
            d = np.abs(st["y"] - start["y"]) + np.abs(st["x"] - start["x"])
            hist = np.bincount(d[movers] * 17 // (L + 1), minlength=17)
            assert a["window"] == L and a["t"] == int(st["counters"][0])
            assert a["population"] == int(alive.sum()) == int(st["counters"][1])
            assert a["resources"] == int(st["res"].sum())
            assert a["movers"] == int(movers.sum())
            np.testing.assert_array_equal(a["move_bins"], hist)
            start = st
    finally:
        gw.close()


def test_batched_windows_equal_alone_windows(eco):
    specs = [(EcoParams(H=20, W=40, n_agents0=60, capacity=240, max_age=70), 4),
             (EcoParams(H=30, W=90, n_agents0=200, capacity=800), 5)]
    worlds = [eco.World(p, s) for p, s in specs]
    alone = [eco.World(p, s) for p, s in specs]
    batch = eco.Batch(worlds)
    for L in (50, 25, 50):
        batch.step(L)
        batch.sync()
        for w, a in zip(worlds, alone):
            a.step(L)
            _same(w.analysis(), a.analysis(), f"window of {L}")
    batch.close()
    for w in worlds + alone:
        w.close()


def test_load_state_starts_a_window(eco):
    p = EcoParams(max_age=60)
    gw = eco.World(p, seed=9)
    gw.step(70)
    st = gw.read_state(weights=(0, p.capacity))
    gw.step(10)
    gw.load_state(st)
    a = gw.analysis()
    pop = int(st["alive"].sum())
    assert a["window"] == 0 and a["t"] == 70 and a["deaths"] == 0
    assert a["movers"] == pop and a["move_bins"][0] == pop
    bad = dict(st)
    bad["age"] = st["age"].copy()
    bad["age"][np.flatnonzero(st["alive"])[0]] = -1
    from paper_2302_09334_gb300._lib import ECO_ESTATE, EcoError
    with pytest.raises(EcoError) as e:
        gw.load_state(bad)
    assert e.value.code == ECO_ESTATE
    gw.close()
