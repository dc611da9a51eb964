"""eco_moves_noalloc: move resolution for callers that cannot allocate.

Some callers of this library cannot call cudaMalloc -- code running under
another allocator that already owns the device's memory, or a loop that must
not stall on an allocation.  eco_moves_noalloc resolves one round of moves
on arrays the caller already owns, with its per-cell claims in a fixed array
inside the library.  This test checks it against the moves the full step
(eco_world_step_forced) makes from the same state with the same actions, on
two calls in a row.  Moves are integer work, so the comparison is exact.

It lives in its own file, named to be collected last, and passes both alone
in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2302_09334_gb300.params import INT32_MAX, EcoParams, paper_200x400

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eco():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    return world


def _held(p: EcoParams) -> EcoParams:
    # no deaths and no births: the agent set stays the same, so positions
    # after a full step are the positions after the moves
    return p.replace(e_decay=0.0, t_repr=INT32_MAX)


@pytest.mark.parametrize("params", [
    _held(EcoParams(H=20, W=40, capacity=256, n_agents0=200)),
    _held(paper_200x400().replace(n_agents0=6000)),
    _held(EcoParams(H=9, W=33, capacity=64, n_agents0=60, border_walls=0)),
])
def test_moves_noalloc_matches_step(eco, params):
    import torch
    from paper_2302_09334_gb300._lib import check, lib

    w = eco.World(params, seed=7)
    st = w.read_state()
    dev = w.device
    H, W, C = params.H, params.W, params.capacity
    as_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    wall = as_dev(st["wall"].astype(np.uint8))
    alive = as_dev(st["alive"])
    y = as_dev(st["y"])
    x = as_dev(st["x"])
    slot_map = as_dev(st["slot_map"])
    killed = torch.zeros(C, dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(3)
    live = st["alive"].astype(bool)
    for call in range(2):
        actions_np = rng.integers(0, 5, C).astype(np.int32)
        actions = as_dev(actions_np)
        w.step_forced(actions_np)
        stream = torch.cuda.current_stream(dev)
        check(lib().eco_moves_noalloc(H, W, C, params.wall_kills,
                                      ctypes.c_void_p(wall.data_ptr()),
                                      ctypes.c_void_p(alive.data_ptr()),
                                      ctypes.c_void_p(actions.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()),
                                      ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(slot_map.data_ptr()),
                                      ctypes.c_void_p(killed.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream)),
              "eco_moves_noalloc")
        torch.cuda.synchronize(dev)
        ref = w.read_state(fields=("alive", "y", "x", "slot_map"))
        np.testing.assert_array_equal(ref["alive"], st["alive"])
        np.testing.assert_array_equal(y.cpu().numpy()[live], ref["y"][live], err_msg=f"call {call}")
        np.testing.assert_array_equal(x.cpu().numpy()[live], ref["x"][live], err_msg=f"call {call}")
        np.testing.assert_array_equal(slot_map.cpu().numpy(), ref["slot_map"],
                                      err_msg=f"call {call}")
        assert not killed.cpu().numpy().any()
    moved = (y.cpu().numpy()[live] != st["y"][live]) | (x.cpu().numpy()[live] != st["x"][live])
    assert moved.sum() > 0


def test_moves_noalloc_wall_kills_match_step(eco):
    """wall_kills = 1: an agent whose move leads into a wall or off the grid
    is flagged in `killed`; the full step removes exactly those agents (and
    no other), and every survivor ends where the full step puts it.  Two
    calls in a row, the second from the state after the first step's
    deaths."""
    import torch
    from paper_2302_09334_gb300._lib import check, lib

    params = _held(EcoParams(H=12, W=30, capacity=128, n_agents0=120, wall_kills=1))
    w = eco.World(params, seed=9)
    st = w.read_state()
    dev = w.device
    H, W, C = params.H, params.W, params.capacity
    as_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    wall_np = st["wall"].astype(np.uint8)
    wall = as_dev(wall_np)
    alive_np = st["alive"].copy()
    y_np, x_np = st["y"].copy(), st["x"].copy()
    alive, y, x = as_dev(alive_np), as_dev(y_np), as_dev(x_np)
    slot_map = as_dev(st["slot_map"])
    killed = torch.zeros(C, dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(4)
    dy, dx = np.array([0, -1, 1, 0, 0]), np.array([0, 0, 0, 1, -1])
    total_killed = 0
    for call in range(2):
        live = alive_np.astype(bool)
        actions_np = rng.integers(0, 5, C).astype(np.int32)
        # agents next to a wall move into it half of the time
        for s in np.flatnonzero(live):
            into = [a for a in range(1, 5)
                    if wall_np[y_np[s] + dy[a], x_np[s] + dx[a]]]
            if into and rng.random() < 0.5:
                actions_np[s] = into[0]
        w.step_forced(actions_np)
        stream = torch.cuda.current_stream(dev)
        check(lib().eco_moves_noalloc(H, W, C, 1, ctypes.c_void_p(wall.data_ptr()),
                                      ctypes.c_void_p(alive.data_ptr()),
                                      ctypes.c_void_p(as_dev(actions_np).data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()),
                                      ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(slot_map.data_ptr()),
                                      ctypes.c_void_p(killed.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream)),
              "eco_moves_noalloc")
        torch.cuda.synchronize(dev)
        ref = w.read_state(fields=("alive", "y", "x", "slot_map"))
        k = killed.cpu().numpy().astype(bool)
        died = live & ~ref["alive"].astype(bool)
        np.testing.assert_array_equal(k & live, died, err_msg=f"call {call}: killed")
        assert not (k & ~live).any()
        surv = live & ~k
        gy, gx = y.cpu().numpy(), x.cpu().numpy()
        np.testing.assert_array_equal(gy[surv], ref["y"][surv], err_msg=f"call {call}")
        np.testing.assert_array_equal(gx[surv], ref["x"][surv], err_msg=f"call {call}")
        # the step also removes the killed agents from the grid
        sm = slot_map.cpu().numpy()
        for s in np.flatnonzero(k):
            sm[gy[s], gx[s]] = -1
        np.testing.assert_array_equal(sm, ref["slot_map"], err_msg=f"call {call}: slot_map")
        total_killed += int(k.sum())
        # the next call starts from the state after the deaths
        alive_np = ref["alive"].copy()
        y_np, x_np = ref["y"].copy(), ref["x"].copy()
        alive.copy_(as_dev(alive_np))
        slot_map.copy_(as_dev(ref["slot_map"]))
    assert total_killed > 0


def test_moves_noalloc_rejects_oversized_grid(eco):
    from paper_2302_09334_gb300._lib import ECO_EINVAL, lib
    rc = lib().eco_moves_noalloc(2048, 1025, 0, 0, None, None, None, None, None, None, None, None)
    assert rc == ECO_EINVAL
