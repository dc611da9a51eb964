"""Comparison of a CUDA world's state with an oracle world's, and the
tolerances of the parity tests.

Tolerances (derived from the arithmetic; see the design notes):
  * grid, positions, slots, counters, energies, reproduction/death
    counters, ages: bit-exact (integer work, and float energies computed by
    the same single IEEE add/sub on both sides);
  * hidden and cell state, logits: |gpu - oracle| <= 1e-5 * E per element,
    E the oracle's error magnitude of that output (or_lstm_mag /
    or_pc_mag: |bias| + sum |w v| of every dot product on its paths,
    carried through the absolute derivatives of the gates, products and
    activations, plus the magnitudes of the step's h and c inputs).  E is
    the scale relative to which an FP32 evaluation is accurate: the GPU's
    dot products of at most 180 terms (4 partial sums of 45 fused
    multiply-adds, a pairwise combine, the bias) err by at most about
    48 * 2^-24 * (|b| + sum |w v|) = 2.9e-6 of it, the activations by a few
    ulp.  For an output whose value is not the result of cancellation E is
    a small multiple of |oracle|, so this is a relative bound; the worst
    true relative error |gpu - oracle| / |oracle| is reported beside it;
  * both sides compute from the same state: after each comparison the
    oracle continues from the GPU's h and c (their magnitudes restart at
    zero), and every agent's weights are the GPU's once checked (the
    initial draw within the weight tolerance of the oracle's, a child's
    mutation within it of the oracle's noise added to the GPU's parent), so
    the RNN check measures one step of the kernel, not drift;
  * weights: each mutation, checked from the GPU's own parent weights
    (w' = w_parent + sigma N_j, noise from the oracle's stream):
    |gpu - expected| <= 1e-6 * (|expected| + sigma); the initial draw
    likewise on the scale of the initial std;
  * actions: equal, except where the oracle's top-two logit margin is below
    1e-5 * (E_first + E_second) (flagged, not counted as a mismatch);
  * sampled actions (the paper's controller): equal, except where the
    agent's uniform lies within tol of a cumulative probability of the
    oracle's softmax at temperature 1/50, tol = 25 * 1e-5 * max_a E_a (a
    logit error d moves a cumulative probability by at most 50 d / 2) +
    2^-24 (100 * (max - min logit) + 16) (the FP32 exponentials).
"""
from __future__ import annotations

import numpy as np

RNN_TOL = 1e-5
W_TOL = 1e-6
U32 = 2.0 ** -24


def rnn_close(gpu, ref, mag, what) -> dict:
    """Assert |gpu - ref| <= RNN_TOL * mag elementwise.  Returns the share of
    the tolerance used (budget) and the worst true relative error."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    mag = np.asarray(mag, np.float64)
    err = np.abs(gpu - ref)
    bound = RNN_TOL * mag
    bad = err > bound
    assert not bad.any(), (f"{what}: {int(bad.sum())} values off, e.g. gpu {gpu[bad][:3]} "
                           f"oracle {ref[bad][:3]} magnitude {mag[bad][:3]}")
    if not err.size:
        return {"budget": 0.0, "rel": 0.0}
    with np.errstate(divide="ignore", invalid="ignore"):
        budget = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0), 0.0)
        rel = np.where(ref != 0, err / np.abs(np.where(ref != 0, ref, 1.0)), 0.0)
    return {"budget": float(budget.max()), "rel": float(rel.max())}


def weights_close(gpu, ref, std, what):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    bound = W_TOL * (np.abs(ref) + std)
    bad = np.abs(gpu - ref) > bound
    assert not bad.any(), (f"{what}: {int(bad.sum())} weights off, max "
                           f"{(np.abs(gpu - ref) / (np.abs(ref) + std)).max():.3g}")


def small_margin(logits, mag):
    """Oracle logits and their magnitudes [n, 5] -> bool [n]: the top-two
    margin is within the logits' tolerance."""
    lg = np.asarray(logits, np.float64)
    mg = np.asarray(mag, np.float64)
    order = np.argsort(-lg, axis=1, kind="stable")
    rows = np.arange(lg.shape[0])
    a, b = order[:, 0], order[:, 1]
    return (lg[rows, a] - lg[rows, b]) <= RNN_TOL * (mg[rows, a] + mg[rows, b])


def sync_weights(gw, ow, slots, std, what, chunk=1024):
    """Check the GPU's weights of `slots` against the oracle's (the initial
    draw or a loaded state: within the weight tolerance on the scale std),
    then give the oracle the GPU's, so that both continue from the same
    weights."""
    slots = np.asarray(slots, np.int64)
    if slots.size == 0:
        return
    n = gw.nparam
    # contiguous runs of slots, read in chunks
    runs = np.split(slots, np.flatnonzero(np.diff(slots) != 1) + 1)
    for run in runs:
        for i in range(0, run.size, chunk):
            first, cnt = int(run[i]), int(min(chunk, run.size - i))
            g = gw.read_state(fields=(), weights=(first, cnt))["weights"]
            weights_close(g, ow.weights[first:first + cnt, :n], std, f"{what} slots {first}..")
            ow.weights[first:first + cnt, :n] = g


def sync_recurrent(gs, ow, live):
    """The oracle continues from the GPU's h and c (exact inputs: their
    magnitudes restart at zero)."""
    ow.h[live] = gs["h"][live]
    ow.c[live] = gs["c"][live]
    ow.mag_h[live] = 0.0
    ow.mag_c[live] = 0.0


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
        stats["h"] = rnn_close(gs["h"][live], ow.h[live], ow.mag_h[live], f"{where}: h")
        stats["c"] = rnn_close(gs["c"][live], ow.c[live], ow.mag_c[live], f"{where}: c")
    return stats


def compare_actions(g_action, g_logits, ow, acted, where: str) -> int:
    """Own argmax and logits of the agents that acted this step; returns
    the number of flagged (small-margin) action differences."""
    idx = np.flatnonzero(acted)
    if idx.size == 0:
        return 0, {"budget": 0.0, "rel": 0.0}
    st = rnn_close(g_logits[idx], ow.logits[idx], ow.mag_logits[idx], f"{where}: logits")
    diff = g_action[idx] != ow.action[idx]
    flagged = small_margin(ow.logits[idx], ow.mag_logits[idx])
    assert not (diff & ~flagged).any(), f"{where}: actions differ at slots {idx[diff & ~flagged]}"
    return int((diff & flagged).sum()), st


def near_sample_boundary(logits, mag, u):
    """Oracle logits and magnitudes [n, 5], uniforms [n] -> bool [n]: u
    within the sampling tolerance of a cumulative probability of
    softmax(50 logits)."""
    lg = np.asarray(logits, np.float64)
    z = np.exp(50.0 * (lg - lg.max(axis=1, keepdims=True)))
    cdf = np.cumsum(z / z.sum(axis=1, keepdims=True), axis=1)[:, :4]
    tol = 25.0 * RNN_TOL * np.asarray(mag, np.float64).max(axis=1) + \
        U32 * (100.0 * (lg.max(axis=1) - lg.min(axis=1)) + 16.0)
    return (np.abs(cdf - np.asarray(u)[:, None]) <= tol[:, None]).any(axis=1)


def compare_sampled_actions(g_action, g_logits, ow, acted, t, where: str) -> int:
    """The paper controller's logits and sampled actions of the agents that
    acted at step t; returns the number of flagged differences."""
    from oracle import pyoracle
    idx = np.flatnonzero(acted)
    if idx.size == 0:
        return 0, {"budget": 0.0, "rel": 0.0}
    st = rnn_close(g_logits[idx], ow.logits[idx], ow.mag_logits[idx], f"{where}: logits")
    u = np.array([pyoracle.action_uniform(ow.seed, t, int(s)) for s in idx])
    diff = g_action[idx] != ow.action[idx]
    flagged = near_sample_boundary(ow.logits[idx], ow.mag_logits[idx], u)
    assert not (diff & ~flagged).any(), f"{where}: sampled actions differ at {idx[diff & ~flagged]}"
    return int((diff & flagged).sum()), st


def _read_rows(gw, slots, chunk=1024):
    """GPU weights of `slots` (logical order), read in runs of consecutive
    slots."""
    slots = np.asarray(slots, np.int64)
    out = np.empty((slots.size, gw.nparam), np.float32)
    order = np.argsort(slots, kind="stable")
    srt = slots[order]
    runs = np.split(np.arange(srt.size), np.flatnonzero(np.diff(srt) != 1) + 1)
    for run in runs:
        for i in range(0, run.size, chunk):
            idx = run[i:i + chunk]
            g = gw.read_state(fields=(), weights=(int(srt[idx[0]]), idx.size))["weights"]
            out[order[idx]] = g
    return out


def check_births(gw, ow, nb, sigma, where, parent_sample=64):
    """Weights of this step's children.  The oracle's parents are the GPU's
    (shared since they were checked), so the oracle's child -- its noise
    stream added to the same parent -- is the expected mutation: every GPU
    child is within the weight tolerance of it, and the oracle continues
    from the GPU's child.  A sample of parents is read back to check that
    they are still the same on both sides."""
    n = gw.nparam
    children = ow.birth_child[:nb].astype(np.int64)
    parents = ow.birth_parent[:nb].astype(np.int64)
    wc = _read_rows(gw, children)
    weights_close(wc, ow.weights[children, :n], sigma, f"{where} children (mutation)")
    ow.weights[children, :n] = wc
    pick = parents if parents.size <= parent_sample else \
        np.random.default_rng(int(ow.counters[0])).choice(parents, parent_sample, replace=False)
    np.testing.assert_array_equal(_read_rows(gw, pick), ow.weights[pick, :n],
                                  err_msg=f"{where}: parents differ from the GPU's")


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
               compare_every: int = 1, init_std: float | None = None) -> dict:
    """Step both worlds `steps` times, the GPU with the actions the oracle
    moved with, and compare after every `compare_every` steps (always after
    births).  The living agents' weights are first checked and shared
    (sync_weights, scale init_std, default the world's initial std); after
    each comparison the oracle continues from the GPU's h and c."""
    flagged = 0
    worst = {"budget": 0.0, "rel": 0.0}
    births = 0
    prev = gw.read_state()
    live0 = np.flatnonzero(ow.alive)
    sync_weights(gw, ow, live0, float(ow.p.w_init_std) if init_std is None else init_std,
                 f"{where} start")
    sync_recurrent(prev, ow, ow.alive.astype(bool))

    def note(st):
        for v in st.values() if "budget" not in st else (st,):
            worst["budget"] = max(worst["budget"], v["budget"])
            worst["rel"] = max(worst["rel"], v["rel"])

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
        note(compare(gs, ow, label))
        # a slot reused by a newborn this step has its action and logits reset
        reborn = np.zeros_like(acted)
        reborn[ow.birth_child[:nb]] = True
        ow_action_saved = ow.action.copy()
        try:
            ow.action[:] = ow.move_action
            if getattr(ow.p, "controller", 0) == 1:
                f, st = compare_sampled_actions(gs["action"], gs["logits"], ow, acted & ~reborn,
                                                int(ow.counters[0]) - 1, label)
            else:
                f, st = compare_actions(gs["action"], gs["logits"], ow, acted & ~reborn, label)
            flagged += f
            note(st)
        finally:
            ow.action[:] = ow_action_saved
        if nb:
            check_births(gw, ow, nb, weight_std, label)
        sync_recurrent(gs, ow, ow.alive.astype(bool))
        prev = gs
    return {"flagged": flagged, "births": births, **worst}


def run_gpu_driven(gw, ow, steps: int, where: str) -> dict:
    """The GPU world runs free, one step at a time; the oracle takes each
    step moving with the actions the GPU took (its own argmax is still
    computed and compared: a difference must be a flagged near-tie), and
    the states are compared after every step under the same rules as
    run_forced, from the same weights and (after each step) the same h and
    c.  An agent that dies in a step whose slot a newborn takes in the same
    step leaves no record of its action; such a step is refused."""
    flagged = 0
    worst = {"budget": 0.0, "rel": 0.0}
    prev = gw.read_state()
    sync_weights(gw, ow, np.flatnonzero(ow.alive), float(ow.p.w_init_std), f"{where} start")
    sync_recurrent(prev, ow, ow.alive.astype(bool))
    for k in range(steps):
        acted = prev["alive"].astype(bool)
        gw.step(1)
        gs = gw.read_state()
        label = f"{where} step {k + 1}"
        reborn = acted & gs["alive"].astype(bool) & (gs["age"] == 0)
        assert not reborn.any(), f"{label}: a slot was reused in the step its agent died"
        forced = np.where(acted, gs["action"], 0).astype(np.int32)
        ow.step(forced)
        for v in compare(gs, ow, label).values():
            worst["budget"] = max(worst["budget"], v["budget"])
            worst["rel"] = max(worst["rel"], v["rel"])
        f, st = compare_actions(gs["action"], gs["logits"], ow, acted, label)
        flagged += f
        worst["budget"] = max(worst["budget"], st["budget"])
        worst["rel"] = max(worst["rel"], st["rel"])
        nb = int(ow.counters[5])
        if nb:
            check_births(gw, ow, nb, float(ow.p.mut_std), label)
        sync_recurrent(gs, ow, ow.alive.astype(bool))
        prev = gs
    return {"flagged": flagged, **worst}
