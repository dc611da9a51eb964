"""Comparison of a CUDA world's state with an oracle world's, and the
tolerances of the parity tests.

Tolerances (derived from the arithmetic; see the design notes):
  * grid, positions, slots, counters, energies, reproduction/death
    counters, ages: bit-exact (integer work, and float energies computed by
    the same single IEEE add/sub on both sides);
  * hidden and cell state, logits: |gpu - oracle| <= 1e-5 * max(1, |oracle|)
    (FP32 on the GPU against FP64 in the oracle; h is in (-1, 1));
  * weights: each mutation, checked from the GPU's own parent weights
    (w' = w_parent + sigma N_j, noise from the oracle's stream):
    |gpu - expected| <= 1e-6 * (|expected| + sigma); and the drift against
    the oracle's child after several generations, relative to the operands
    of the mutation and scaled by the child's generation g (each mutation
    adds its own rounding, the initial draw one more, on the scale of the
    initial weights' std sigma0):
    |gpu - oracle| <= 1e-6 (g (|oracle| + |parent| + sigma)
                            + |oracle| + |parent| + sigma0);
  * actions: equal, except where the oracle's top-two logit margin is below
    1e-5 * max(1, max|logit|) (flagged, not counted as a mismatch);
  * sampled actions (the paper's controller): equal, except where the
    agent's uniform lies within 2e-3 * max(1, max|logit|) of a cumulative
    probability of the oracle's softmax at temperature 1/50 (the logit
    tolerance, scaled by 50 for the two logits of a difference, bounds the
    error of every cumulative probability by 1e-3 * max(1, max|logit|)).
"""
from __future__ import annotations

import numpy as np

RNN_TOL = 1e-5
W_TOL = 1e-6
SAMPLE_TOL = 2e-3


def rnn_close(gpu, ref, what):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(gpu - ref) / np.maximum(1.0, np.abs(ref))
    bad = err > RNN_TOL
    assert not bad.any(), f"{what}: {int(bad.sum())} values off, max rel {err.max():.3g}"
    return float(err.max()) if err.size else 0.0


def weights_close(gpu, ref, std, what):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    bound = W_TOL * (np.abs(ref) + std)
    bad = np.abs(gpu - ref) > bound
    assert not bad.any(), (f"{what}: {int(bad.sum())} weights off, max "
                           f"{(np.abs(gpu - ref) / (np.abs(ref) + std)).max():.3g}")


def weights_drift_close(gpu, ref, parent, std, generation, what, init_std=None):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    mag = np.abs(ref) + np.abs(np.asarray(parent, np.float64))
    # each mutation adds its rounding; the initial draw one more, on the
    # scale of the initial weights
    bound = W_TOL * (generation * (mag + std) + mag + (std if init_std is None else init_std))
    bad = np.abs(gpu - ref) > bound
    assert not bad.any(), f"{what}: {int(bad.sum())} weights drifted"


def small_margin(logits):
    """Oracle logits [n, 5] -> bool [n]: top-two margin below tolerance."""
    lg = np.asarray(logits, np.float64)
    s = np.sort(lg, axis=1)
    return (s[:, -1] - s[:, -2]) < RNN_TOL * np.maximum(1.0, np.abs(lg).max(axis=1))


def compare(gs: dict, ow, where: str, check_rnn: bool = True) -> dict:
    """Assert the GPU state equals the oracle's (rules above).  Returns stats."""
    np.testing.assert_array_equal(gs["counters"], ow.counters, err_msg=f"{where}: counters")
    np.testing.assert_array_equal(gs["res"], ow.res, err_msg=f"{where}: res")
    np.testing.assert_array_equal(gs["wall"], ow.wall, err_msg=f"{where}: wall")
    np.testing.assert_array_equal(gs["alive"], ow.alive, err_msg=f"{where}: alive")
    np.testing.assert_array_equal(gs["slot_map"], ow.slot_map, err_msg=f"{where}: slot_map")
    live = ow.alive.astype(bool)
    for f in ("y", "x", "repr_ctr", "low_ctr", "age", "prev_action", "ate"):
        np.testing.assert_array_equal(gs[f][live], getattr(ow, f)[live], err_msg=f"{where}: {f}")
    np.testing.assert_array_equal(gs["energy"][live].view(np.uint32),
                                  ow.energy[live].view(np.uint32), err_msg=f"{where}: energy")
    stats = {}
    if check_rnn and live.any():
        stats["h"] = rnn_close(gs["h"][live], ow.h[live], f"{where}: h")
        stats["c"] = rnn_close(gs["c"][live], ow.c[live], f"{where}: c")
    return stats


def compare_actions(g_action, g_logits, ow, acted, where: str) -> int:
    """Own argmax and logits of the agents that acted this step; returns
    the number of flagged (small-margin) action differences."""
    idx = np.flatnonzero(acted)
    if idx.size == 0:
        return 0
    rnn_close(g_logits[idx], ow.logits[idx], f"{where}: logits")
    diff = g_action[idx] != ow.action[idx]
    flagged = small_margin(ow.logits[idx])
    assert not (diff & ~flagged).any(), f"{where}: actions differ at slots {idx[diff & ~flagged]}"
    return int((diff & flagged).sum())


def near_sample_boundary(logits, u):
    """Oracle logits [n, 5], uniforms [n] -> bool [n]: u within the sampling
    tolerance of a cumulative probability of softmax(50 logits)."""
    lg = np.asarray(logits, np.float64)
    z = np.exp(50.0 * (lg - lg.max(axis=1, keepdims=True)))
    cdf = np.cumsum(z / z.sum(axis=1, keepdims=True), axis=1)[:, :4]
    tol = SAMPLE_TOL * np.maximum(1.0, np.abs(lg).max(axis=1))
    return (np.abs(cdf - np.asarray(u)[:, None]) < tol[:, None]).any(axis=1)


def compare_sampled_actions(g_action, g_logits, ow, acted, t, where: str) -> int:
    """The paper controller's logits and sampled actions of the agents that
    acted at step t; returns the number of flagged differences."""
    from oracle import pyoracle
    idx = np.flatnonzero(acted)
    if idx.size == 0:
        return 0
    rnn_close(g_logits[idx], ow.logits[idx], f"{where}: logits")
    u = np.array([pyoracle.action_uniform(ow.seed, t, int(s)) for s in idx])
    diff = g_action[idx] != ow.action[idx]
    flagged = near_sample_boundary(ow.logits[idx], u)
    assert not (diff & ~flagged).any(), f"{where}: sampled actions differ at {idx[diff & ~flagged]}"
    return int((diff & flagged).sum())


def check_births(gw, ow, nb, sigma, where, gen):
    """Weights of this step's children (see the tolerance rules above);
    gen[slot] is the generation of the agent in the slot (updated here)."""
    from oracle import pyoracle
    t = int(ow.counters[0]) - 1
    parents = ow.birth_parent[:nb].copy()
    children = ow.birth_child[:nb].copy()
    for par, ch in zip(parents, children):
        wp = gw.read_state(fields=(), weights=(int(par), 1))["weights"][0]
        wc = gw.read_state(fields=(), weights=(int(ch), 1))["weights"][0]
        n = wp.shape[0]
        expected = pyoracle.fill_normals_n(ow.seed, pyoracle.TAG_MUT, t, int(par), sigma, n, wp)
        weights_close(wc, expected, sigma, f"{where} child {ch} (mutation)")
        gen[ch] = gen[par] + 1
        weights_drift_close(wc, ow.weights[ch, :n], ow.weights[par, :n], sigma, gen[ch],
                            f"{where} child {ch} (generation {gen[ch]})",
                            init_std=float(ow.p.w_init_std))


def _diagnose(prev, gs, ow, forced, where):
    """Describe the agents around every cell where the slot maps differ."""
    lines = [f"{where}: slot_map differs"]
    cells = np.argwhere(gs["slot_map"] != ow.slot_map)
    near = set()
    for (y, x) in cells:
        for s in (int(gs["slot_map"][y, x]), int(ow.slot_map[y, x])):
            if s >= 0:
                near.add(s)
        for s in np.flatnonzero(prev["alive"]):
            if abs(int(prev["y"][s]) - y) + abs(int(prev["x"][s]) - x) <= 2:
                near.add(int(s))
    for s in sorted(near):
        lines.append(
            f"  slot {s}: before ({prev['y'][s]},{prev['x'][s]}) alive {prev['alive'][s]} "
            f"forced {forced[s]} gpu_action {gs['action'][s]} oracle_move {ow.move_action[s]} "
            f"after gpu ({gs['y'][s]},{gs['x'][s]}) alive {gs['alive'][s]} "
            f"oracle ({ow.y[s]},{ow.x[s]}) alive {ow.alive[s]}")
    lines.append(f"  births {ow.birth_parent[:ow.counters[5]]} -> {ow.birth_child[:ow.counters[5]]}")
    return "\n".join(lines)


def run_forced(gw, ow, steps: int, where: str, weight_std: float,
               compare_every: int = 1) -> dict:
    """Step both worlds `steps` times, the GPU with the actions the oracle
    moved with, and compare after every `compare_every` steps (always after
    births)."""
    flagged = 0
    worst = {"h": 0.0, "c": 0.0}
    births = 0
    prev = gw.read_state()
    gen = np.zeros(ow.p.capacity, np.int64)   # loaded/initial agents: generation 0
    for k in range(steps):
        acted = ow.alive.copy().astype(bool)
        ow.step()
        forced = ow.move_action.copy()
        gw.step_forced(forced)
        nb = int(ow.counters[5])
        births += nb
        if (k + 1) % compare_every and nb == 0 and k != steps - 1:
            continue
        gs = gw.read_state()
        label = f"{where} step {k + 1}"
        if not np.array_equal(gs["slot_map"], ow.slot_map):
            raise AssertionError(_diagnose(prev, gs, ow, forced, label))
        st = compare(gs, ow, label)
        for key in st:
            worst[key] = max(worst[key], st[key])
        # a slot reused by a newborn this step has its action and logits reset
        reborn = np.zeros_like(acted)
        reborn[ow.birth_child[:nb]] = True
        ow_action_saved = ow.action.copy()
        try:
            ow.action[:] = ow.move_action
            if getattr(ow.p, "controller", 0) == 1:
                flagged += compare_sampled_actions(gs["action"], gs["logits"], ow,
                                                   acted & ~reborn, int(ow.counters[0]) - 1,
                                                   label)
            else:
                flagged += compare_actions(gs["action"], gs["logits"], ow, acted & ~reborn,
                                           label)
        finally:
            ow.action[:] = ow_action_saved
        if nb:
            check_births(gw, ow, nb, weight_std, label, gen)
        prev = gs
    return {"flagged": flagged, "births": births, **worst}
