"""Lab-environment greediness on the GPU (App. C): the windows with a
resource in view (T_r) and with a meal (C_r) equal the oracle's, slot for
slot, on forced runs of both controllers, and in a lab world (one agent,
no regrowth, no reproduction) holding an agent evolved in a natural world."""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams, lab
from tests.parity import run_forced

pytestmark = pytest.mark.gpu

WINDOW = 20


@pytest.fixture(scope="module")
def eco():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    return world


def _check(gw, ow, where):
    T, C = gw.lab_read()
    live = ow.alive.astype(bool)
    np.testing.assert_array_equal(T[live], ow.lab_t[live], err_msg=f"{where}: T_r")
    np.testing.assert_array_equal(C[live], ow.lab_c[live], err_msg=f"{where}: C_r")
    assert np.all(C[live] <= T[live])
    return int(T[live].sum()), int(C[live].sum())


@pytest.mark.parametrize("controller", [0, 1])
def test_lab_counters_equal_oracle(eco, oracle, controller):
    p = EcoParams(H=24, W=48, capacity=300, n_agents0=80, t_repr=40, e_repr=0.6,
                  max_age=150, controller=controller, w_init_std=0.5)
    gw = eco.World(p, seed=12)
    ow = oracle.OracleWorld(p.asdict(), 12)
    tot_t = tot_c = 0
    for w in range(6):
        run_forced(gw, ow, WINDOW, f"ctrl {controller} window {w}", p.mut_std,
                   compare_every=WINDOW)
        gw.lab_window()
        ow.lab_window()
        tot_t, tot_c = _check(gw, ow, f"ctrl {controller} window {w}")
    assert tot_t > 0 and tot_c > 0
    gw.close()
    ow.close()


@pytest.mark.parametrize("density", [0.05, 0.3])
def test_lab_world_with_an_evolved_agent(eco, oracle, density):
    nat = EcoParams(H=30, W=60, capacity=400, n_agents0=120, t_repr=30, e_repr=0.5)
    src = eco.World(nat, seed=3)
    src.step(120)
    st = src.read_state(fields=("alive", "age"), weights=(0, nat.capacity))
    alive = np.flatnonzero(st["alive"])
    s_old = int(alive[np.argmax(st["age"][alive])])      # the oldest agent
    w_evolved = st["weights"][s_old].copy()
    src.close()

    p = lab(nat, density)
    gw = eco.World(p, seed=5)
    ow = oracle.OracleWorld(p.asdict(), 5)
    ls = gw.read_state(weights=(0, 1))
    ls["weights"] = w_evolved[None]
    gw.load_state(ls)
    ow.weights[0, :w_evolved.shape[0]] = w_evolved
    ow.sync()
    for w in range(10):
        run_forced(gw, ow, WINDOW, f"lab {density} window {w}", p.mut_std,
                   compare_every=WINDOW)
        gw.lab_window()
        ow.lab_window()
        _check(gw, ow, f"lab {density} window {w}")
    assert int(ow.counters[2]) == 0                     # no reproduction in the lab
    gw.close()
    ow.close()
