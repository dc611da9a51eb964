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
    of the mutation: |gpu - oracle| <= 1e-6 * (|oracle| + |parent| + sigma)
    (each generation may round the parent differently by one ulp);
  * actions: equal, except where the oracle's top-two logit margin is below
    1e-5 * max(1, max|logit|) (flagged, not counted as a mismatch).
"""
from __future__ import annotations

import numpy as np

RNN_TOL = 1e-5
W_TOL = 1e-6


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


def weights_drift_close(gpu, ref, parent, std, what):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    bound = W_TOL * (np.abs(ref) + np.abs(np.asarray(parent, np.float64)) + std)
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
    for f in ("y", "x", "repr_ctr", "low_ctr", "age"):
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


def check_births(gw, ow, nb, sigma, where):
    """Weights of this step's children (see the tolerance rules above)."""
    from oracle import pyoracle
    t = int(ow.counters[0]) - 1
    parents = ow.birth_parent[:nb].copy()
    children = ow.birth_child[:nb].copy()
    for par, ch in zip(parents, children):
        wp = gw.read_state(fields=(), weights=(int(par), 1))["weights"][0]
        wc = gw.read_state(fields=(), weights=(int(ch), 1))["weights"][0]
        expected = pyoracle.fill_normals(ow.seed, pyoracle.TAG_MUT, t, int(par), sigma, wp)
        weights_close(wc, expected, sigma, f"{where} child {ch} (mutation)")
        weights_drift_close(wc, ow.weights[ch], ow.weights[par], sigma, f"{where} child {ch}")


def run_forced(gw, ow, steps: int, where: str, weight_std: float,
               compare_every: int = 1) -> dict:
    """Step both worlds `steps` times, the GPU with the oracle's actions, and
    compare after every `compare_every` steps (always after births)."""
    C = ow.p.capacity
    flagged = 0
    worst = {"h": 0.0, "c": 0.0}
    births = 0
    for k in range(steps):
        acted = ow.alive.copy().astype(bool)
        ow.step()
        forced = np.where(acted, ow.action, 0).astype(np.int32)
        gw.step_forced(forced)
        nb = int(ow.counters[5])
        births += nb
        if (k + 1) % compare_every and nb == 0 and k != steps - 1:
            continue
        gs = gw.read_state()
        st = compare(gs, ow, f"{where} step {k + 1}")
        for key in st:
            worst[key] = max(worst[key], st[key])
        flagged += compare_actions(gs["action"], gs["logits"], ow, acted, f"{where} step {k + 1}")
        if nb:
            check_births(gw, ow, nb, weight_std, f"{where} step {k + 1}")
    assert C >= 0
    return {"flagged": flagged, "births": births, **worst}
