"""Seeded synthetic world states, loaded into both the oracle and the CUDA
library by the parity tests.  This module draws inputs only (numpy's PCG64
generator); it computes nothing of the simulation step.

A state has walls (border ring plus random interior walls), resources on
non-wall cells, agents on distinct non-wall cells in random slots, float32
energies spread around the reproduction and death thresholds, counters,
recurrent state and weights ~ N(0, std^2) like freshly initialised agents.
"""
from __future__ import annotations

import numpy as np

NPARAM = 23333


def random_state(p, seed: int, n_agents: int | None = None, wall_p: float = 0.03,
                 res_p: float = 0.15, w_std: float = 0.1, t: int = 0,
                 near_thresholds: bool = True) -> dict:
    rng = np.random.default_rng(seed)
    H, W, C = p.H, p.W, p.capacity
    wall = np.zeros((H, W), np.uint8)
    if p.border_walls:
        wall[0, :] = wall[-1, :] = wall[:, 0] = wall[:, -1] = 1
    wall[rng.random((H, W)) < wall_p] = 1
    res = ((rng.random((H, W)) < res_p) & (wall == 0)).astype(np.uint8)
    free = np.flatnonzero(wall.ravel() == 0)
    if n_agents is None:
        n_agents = min(C, len(free)) // 2
    n_agents = min(n_agents, C, len(free))
    cells = rng.choice(free, n_agents, replace=False)
    slots = np.sort(rng.choice(C, n_agents, replace=False))
    alive = np.zeros(C, np.uint8)
    alive[slots] = 1
    y = np.zeros(C, np.int32)
    x = np.zeros(C, np.int32)
    y[slots] = cells // W
    x[slots] = cells % W
    if near_thresholds:
        e = rng.choice(np.array([p.e_decay, p.e_repr, p.e_repr + p.e_decay, 1.0, 0.3],
                                np.float32), C)
        e = (e + rng.integers(-2, 3, C).astype(np.float32) * np.float32(1e-7)).astype(np.float32)
    else:
        e = rng.uniform(0.05, 1.5, C).astype(np.float32)
    energy = np.where(alive == 1, e, np.float32(0)).astype(np.float32)
    t_repr = int(min(p.t_repr, 10**6))
    repr_ctr = np.where(alive == 1, rng.integers(0, max(t_repr, 1) + 1, C), 0).astype(np.int32)
    low_ctr = np.zeros(C, np.int32)
    age = np.where(alive == 1, rng.integers(0, 500, C), 0).astype(np.int32)
    h = np.where(alive[:, None] == 1, rng.uniform(-0.9, 0.9, (C, 32)), 0).astype(np.float32)
    c = np.where(alive[:, None] == 1, rng.uniform(-2, 2, (C, 32)), 0).astype(np.float32)
    weights = (rng.standard_normal((C, NPARAM)) * w_std).astype(np.float32)
    counters = np.zeros(9, np.int64)
    counters[0] = t
    return dict(res=res, wall=wall, alive=alive, y=y, x=x, energy=energy,
                repr_ctr=repr_ctr, low_ctr=low_ctr, age=age, h=h, c=c,
                action=np.zeros(C, np.int32), logits=np.zeros((C, 5), np.float32),
                weights=weights, counters=counters)


def load_into_oracle(ow, state: dict) -> None:
    """Write a state into an oracle world (its fields are numpy views)."""
    ow.res[:] = state["res"]
    ow.wall[:] = state["wall"]
    ow.alive[:] = state["alive"]
    ow.y[:] = state["y"]
    ow.x[:] = state["x"]
    ow.energy[:] = state["energy"]
    ow.repr_ctr[:] = state["repr_ctr"]
    ow.low_ctr[:] = state["low_ctr"]
    ow.age[:] = state["age"]
    ow.h[:] = state["h"].astype(np.float64)
    ow.c[:] = state["c"].astype(np.float64)
    ow.weights[:] = state["weights"]
    ow.counters[:] = 0
    ow.counters[0] = state["counters"][0]
    ow.sync()
