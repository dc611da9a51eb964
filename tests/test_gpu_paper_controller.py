"""The paper's controller (App. B.5) on the GPU against the oracle:
initial state, forced runs compared step by step (view, CNN, LSTM(4),
dense layers, sampled actions, previous-action and ate inputs, mutation of
the 2445 parameters), the natural-environment preset, batches, and state
I/O round trips."""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams, paper_natural
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


SMALL = EcoParams(H=30, W=60, capacity=400, n_agents0=100, controller=1, e0=3.0, e_max=3.0,
                  e_decay=0.025, e_gain=1.0, e_repr=0.0, t_repr=30, e_death=0.0, t_death=20,
                  max_age=90, res_init_p=0.2, wall_kills=1, w_init_std=0.5)


def test_initial_state(eco, oracle):
    gw = eco.World(SMALL, seed=4)
    ow = oracle.OracleWorld(SMALL.asdict(), 4)
    st = gw.read_state(weights=(0, SMALL.n_agents0))
    compare(st, ow, "init")
    assert st["weights"].shape == (SMALL.n_agents0, 2445)
    weights_close(st["weights"][7], ow.weights[7, :2445], SMALL.w_init_std, "initial weights")
    assert not st["prev_action"].any() and not st["ate"].any()
    gw.close()


def test_forced_run_small(eco, oracle):
    gw = eco.World(SMALL, seed=4)
    ow = oracle.OracleWorld(SMALL.asdict(), 4)
    st = run_forced(gw, ow, 150, "paper small", SMALL.mut_std)
    c = ow.counters
    assert c[2] > 0 and c[3] > 0, "births and deaths expected"
    assert st["flagged"] <= 5
    gw.close()


def test_forced_run_paper_preset(eco, oracle):
    p = paper_natural()
    gw = eco.World(p, seed=0)
    ow = oracle.OracleWorld(p.asdict(), 0)
    st = run_forced(gw, ow, 40, "paper preset", p.mut_std, compare_every=10)
    assert st["flagged"] <= 5
    gw.close()


def test_batch_equals_alone_and_mixing_refused(eco):
    from paper_2302_09334_gb300._lib import ECO_EINVAL, EcoError
    specs = [(SMALL, 1), (SMALL.replace(H=20, W=45, n_agents0=50, capacity=200), 2)]
    worlds = [eco.World(p, s) for p, s in specs]
    batch = eco.Batch(worlds)
    batch.step(60)
    batch.sync()
    for (p, s), w in zip(specs, worlds):
        alone = eco.World(p, s)
        alone.step(60)
        a, b = alone.read_state(weights=(0, p.capacity)), w.read_state(weights=(0, p.capacity))
        live = a["alive"].astype(bool)
        for k in a:
            # slots never used hold whatever the arena held: compare the living
            per_slot = a[k].shape[:1] == (p.capacity,) and k not in ("res", "wall", "slot_map")
            np.testing.assert_array_equal(a[k][live] if per_slot else a[k],
                                          b[k][live] if per_slot else b[k],
                                          err_msg=f"world {s} {k}")
        alone.close()
    batch.close()
    lstm = eco.World(EcoParams(), seed=0)
    with pytest.raises(EcoError) as e:
        eco.Batch([worlds[0], lstm])
    assert e.value.code == ECO_EINVAL
    for w in worlds + [lstm]:
        w.close()


def test_state_round_trip(eco, oracle):
    gw = eco.World(SMALL, seed=8)
    gw.step(45)
    st = gw.read_state(weights=(0, SMALL.capacity))
    assert st["prev_action"][st["alive"].astype(bool)].any()
    other = eco.World(SMALL, seed=8)
    other.load_state(st)
    gw.step(20)
    other.step(20)
    a = gw.read_state(weights=(0, SMALL.capacity))
    b = other.read_state(weights=(0, SMALL.capacity))
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    gw.close()
    other.close()
