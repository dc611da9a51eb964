"""World parameters and the named workloads.

`EcoParams` mirrors the C struct of the library header field for field; the
presets are the synthetic worlds shaped like the paper's natural environment
(App. B.4 hyper-parameters: a 200x400 grid, thousands of agents, runs meant
for 10^6 steps) at three scales.
"""
from __future__ import annotations

import dataclasses
import math

INT32_MAX = 2**31 - 1


@dataclasses.dataclass
class EcoParams:
    H: int = 20
    W: int = 40
    capacity: int = 256
    n_agents0: int = 64
    border_walls: int = 1
    res_init_p: float = 0.1
    nbr_shape: int = 0            # 0: square (Chebyshev) radius, 1: diamond
    nbr_radius: int = 2
    class_edges: tuple = (1, 3, 5)  # classes 0 | 1-2 | 3-4 | >=5
    p_class: tuple = (0.0, 0.001, 0.005, 0.025)
    lat_mode: int = 0             # 0: linear, 1: (alpha^x + 1)/(alpha + 1)
    lat_top: float = 0.2
    lat_bottom: float = 1.0
    lat_alpha: float = 200.0
    p_spont: float = 1e-5
    e0: float = 1.0
    e_decay: float = 0.01
    e_gain: float = 0.2
    e_max: float = math.inf
    e_repr: float = 0.5
    t_repr: int = 50
    e_death: float = 0.0
    t_death: int = 0
    max_age: int = INT32_MAX
    wall_kills: int = 0
    w_init_std: float = 0.1
    mut_std: float = 0.02
    controller: int = 0           # 0: LSTM(32) on the 7x7 view + energy, argmax;
                                  # 1: the paper's CNN -> LSTM(4) -> dense, sampled (App. B.5)

    def replace(self, **kw) -> "EcoParams":
        return dataclasses.replace(self, **kw)

    def asdict(self) -> dict:
        return dataclasses.asdict(self)


def small_20x40() -> EcoParams:
    """20x40 grid, 64 agents (capacity 256); the parity world."""
    return EcoParams()


def paper_200x400() -> EcoParams:
    """Paper-scale 200x400 grid (App. B.4), 1000 agents, capacity 8192."""
    return EcoParams(H=200, W=400, capacity=8192, n_agents0=1000)


def large_1000x2000() -> EcoParams:
    """1000x2000 grid, 20,000 agents, capacity 131,072 (12.2 GB of weights)."""
    return EcoParams(H=1000, W=2000, capacity=131072, n_agents0=20000)


def paper_natural() -> EcoParams:
    """The paper's natural environment (App. B.4, B.5): 200x400 grid, 330
    agents at the start, at most 1000, the CNN+LSTM(4) controller with its
    15x15 view and sampled actions, von Neumann regrowth (p = 0.002 when
    exactly one of the 4 direct neighbours holds a resource) scaled by the
    climate (200^x + 1)/201 plus 5e-5, ~16,000 initial resources, E0 = Emax
    = 3, decay 0.025, gain 1, reproduction after 140 steps above 0, death
    after 200 steps at or below 0 or past age 650, walls that kill."""
    return EcoParams(H=200, W=400, capacity=1000, n_agents0=330, res_init_p=0.2,
                     nbr_shape=1, nbr_radius=1, class_edges=(1, 2, 5),
                     p_class=(0.0, 0.002, 0.0, 0.0), lat_mode=1, lat_alpha=200.0,
                     p_spont=5e-5, e0=3.0, e_max=3.0, e_decay=0.025, e_gain=1.0,
                     e_repr=0.0, t_repr=140, e_death=0.0, t_death=200, max_age=650,
                     wall_kills=1, controller=1)


def lab(p: EcoParams, res_init_p: float, reproduction: bool = False,
        capacity: int = 1) -> EcoParams:
    """Lab environment of the paper's greediness study (App. C): the world
    of `p` with one agent, resource regrowth switched off, initial resources
    Bernoulli(res_init_p), and reproduction off unless asked for (then up
    to `capacity` agents).  Load the evolved agent into slot 0 with
    World.load_state; greediness comes from World.lab_window/lab_read."""
    return p.replace(n_agents0=1, capacity=max(1, capacity), res_init_p=res_init_p,
                     p_class=(0.0, 0.0, 0.0, 0.0), p_spont=0.0,
                     t_repr=p.t_repr if reproduction else INT32_MAX)


def held(p: EcoParams) -> EcoParams:
    """Held population: no energy decay and no reproduction, so the agent
    count stays at n_agents0 (roofline microbenchmark)."""
    return p.replace(e_decay=0.0, t_repr=INT32_MAX)


PRESETS = {
    "small_20x40": small_20x40,
    "paper_200x400": paper_200x400,
    "large_1000x2000": large_1000x2000,
    "paper_natural": paper_natural,
}


# ---------------------------------------------------------------------------
# Many-world workloads.  Their shapes are drawn from a host Philox stream
# (numpy's Philox bit generator, seed 12345) so that runs are reproducible;
# these draws are inputs, not part of the simulation.
# ---------------------------------------------------------------------------
def _host_rng(seed: int = 12345):
    import numpy as np
    return np.random.Generator(np.random.Philox(seed))


def batched_64(n_worlds: int = 64, seed: int = 12345) -> list:
    """64 independent worlds stepped in one launch per kernel: grid sides
    log-uniform between 50x100 and 200x400 (aspect 1:2), initial populations
    uniform in 100..4000, capacity 4x the initial population, bottom-row
    climate factor uniform in [0.5, 1.0] (top 0.2).  World i uses seed i.
    Returns [(EcoParams, seed)]."""
    import math
    rng = _host_rng(seed)
    out = []
    for i in range(n_worlds):
        h = int(round(math.exp(rng.uniform(math.log(50), math.log(200)))))
        n0 = int(rng.integers(100, 4001))
        free = (h - 2) * (2 * h - 2)
        n0 = min(n0, free // 2)
        p = EcoParams(H=h, W=2 * h, n_agents0=n0, capacity=4 * n0,
                      lat_bottom=float(rng.uniform(0.5, 1.0)))
        out.append((p, i))
    return out


SERVE_GRIDS = ((50, 100), (100, 200), (200, 400))


def serve_trace(rate_per_s: float = 20.0, duration_s: float = 600.0, seed: int = 12345) -> list:
    """Simulation requests with Poisson arrivals: grid one of 50x100,
    100x200, 200x400; initial population uniform in 200..3000 (at most half
    the free cells); capacity 4x; steps uniform in 1000..20000; request k
    uses seed k.  Returns [dict(arrival, params, seed, steps)]."""
    rng = _host_rng(seed)
    out, t, k = [], 0.0, 0
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            break
        h, w = SERVE_GRIDS[int(rng.integers(0, len(SERVE_GRIDS)))]
        n0 = min(int(rng.integers(200, 3001)), (h - 2) * (w - 2) // 2)
        steps = int(rng.integers(1000, 20001))
        p = EcoParams(H=h, W=w, n_agents0=n0, capacity=4 * n0)
        out.append({"arrival": t, "params": p, "seed": k, "steps": steps})
        k += 1
    return out
