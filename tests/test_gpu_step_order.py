"""A step starts with the kernel that regrows the step's plane and mutates
the previous step's births; a state read that returns weights first does
that mutation for the pending births.  Reads between steps must change
nothing: a world read after every chunk (all weights, a few rows, counters
only) and a world never read until the end hold the same state, bit for
bit, and a state loaded between steps continues the same way."""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams

pytestmark = pytest.mark.gpu

P = EcoParams(H=30, W=60, capacity=600, n_agents0=150, t_repr=25, e_repr=0.4, max_age=140)


@pytest.fixture(scope="module")
def eco():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    return world


def _state(w):
    """Full state; per-slot fields and weights of living agents only (rows
    of slots never used hold whatever the arena held)."""
    st = w.read_state(weights=(0, P.capacity))
    live = st["alive"].astype(bool)
    st["weights"] = st["weights"][live]
    for f in ("h", "c", "logits", "y", "x", "energy", "repr_ctr", "low_ctr", "age", "action"):
        st[f] = st[f][live]
    return st


def _equal(a, b, where):
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=f"{where}: {k}")


@pytest.mark.parametrize("fused", [1, 0])
def test_reads_between_steps_change_nothing(eco, fused):
    read, plain = eco.World(P, seed=31), eco.World(P, seed=31)
    for w in (read, plain):
        w.set_config(fused=fused, steps_per_graph=4)
    # up to a step with births, whose weights are then pending
    for _ in range(100):
        read.step(1)
        plain.step(1)
        if int(read.counters()[5]) > 0:
            break
    assert int(read.counters()[5]) > 0
    births = 0
    for i, n in enumerate((0, 1, 1, 24, 13, 50, 7)):
        read.step(n)
        plain.step(n)
        if i % 3 == 0:
            st = read.read_state(weights=(0, P.capacity))
        elif i % 3 == 1:
            st = read.read_state(weights=(0, 10))
        else:
            st = read.read_state(fields=())
        births = int(st["counters"][2])
    assert births > 0
    _equal(_state(plain), _state(read), "after the chunks")
    read.close()
    plain.close()


def test_state_loaded_between_steps_continues_the_same(eco):
    a, b = eco.World(P, seed=7), eco.World(P, seed=7)
    for _ in range(100):                        # up to a step with births
        a.step(1)
        if int(a.counters()[5]) > 0:
            break
    st = a.read_state(weights=(0, P.capacity))  # their weights were pending
    assert int(st["counters"][5]) > 0
    b.load_state(st)
    a.step(40)
    b.step(40)
    _equal(_state(a), _state(b), "loaded world")
    a.close()
    b.close()
