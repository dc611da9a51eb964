"""Pins of the oracle's observation and controller (App. B.2).

* observation: rebuilt from padded numpy slices of the three channels;
* LSTM step: torch.nn.LSTMCell in float64 with the same weights (gate order
  i, f, g, o), and a closed form when only the biases are non-zero.
"""
import numpy as np
import pytest
import torch

from paper_2302_09334_gb300.params import EcoParams


def _obs_by_slicing(res, wall, slot_map, y, x, energy):
    pad = 3
    r = np.pad(res, pad, constant_values=0)
    a = np.pad((slot_map >= 0).astype(np.uint8), pad, constant_values=0)
    w = np.pad(wall, pad, constant_values=1)
    win = lambda m: m[y:y + 7, x:x + 7].astype(np.float64).copy()  # noqa: E731
    ra, aa, wa = win(r), win(a), win(w)
    aa[3, 3] = 0.0  # the agent itself is not "another agent"
    return np.concatenate([ra.ravel(), aa.ravel(), wa.ravel(), [np.float32(energy)]])


def test_observe_matches_slicing(oracle):
    rng = np.random.default_rng(3)
    p = EcoParams(H=13, W=21)
    res = (rng.random((p.H, p.W)) < 0.4).astype(np.uint8)
    wall = (rng.random((p.H, p.W)) < 0.2).astype(np.uint8)
    slot_map = np.where(rng.random((p.H, p.W)) < 0.3, rng.integers(0, 50, (p.H, p.W)), -1).astype(np.int32)
    for (y, x) in [(0, 0), (12, 20), (6, 10), (2, 19), (11, 1), (3, 3)]:
        e = np.float32(rng.random())
        got = oracle.observe(p.asdict(), res, wall, slot_map, y, x, e)
        want = _obs_by_slicing(res, wall, slot_map, y, x, e)
        np.testing.assert_array_equal(got, want)


def _torch_lstm(w, obs, h, c):
    cell = torch.nn.LSTMCell(148, 32).double()
    W = torch.tensor(w[:23040].reshape(128, 180), dtype=torch.float64)
    with torch.no_grad():
        cell.weight_ih.copy_(W[:, :148])
        cell.weight_hh.copy_(W[:, 148:])
        cell.bias_ih.copy_(torch.tensor(w[23040:23168], dtype=torch.float64))
        cell.bias_hh.zero_()
        h2, c2 = cell(torch.tensor(obs)[None], (torch.tensor(h)[None], torch.tensor(c)[None]))
        Wo = torch.tensor(w[23168:23328].reshape(5, 32), dtype=torch.float64)
        bo = torch.tensor(w[23328:23333], dtype=torch.float64)
        logits = torch.nn.functional.linear(h2, Wo, bo)
    return h2[0].numpy(), c2[0].numpy(), logits[0].numpy()


def test_lstm_matches_torch_lstmcell(oracle):
    rng = np.random.default_rng(4)
    for trial in range(5):
        w = (rng.standard_normal(23333) * 0.1).astype(np.float32)
        obs = rng.integers(0, 2, 148).astype(np.float64)
        obs[147] = rng.random()
        h = rng.uniform(-1, 1, 32)
        c = rng.uniform(-2, 2, 32)
        a, h2, c2, logits = oracle.lstm_step(w, obs, h, c)
        th, tc, tl = _torch_lstm(w, obs, h, c)
        np.testing.assert_allclose(h2, th, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(c2, tc, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(logits, tl, rtol=1e-12, atol=1e-14)
        assert a == int(np.argmax(tl))


def test_lstm_bias_only_closed_form(oracle):
    sig = lambda z: 1.0 / (1.0 + np.exp(-np.float64(z)))  # noqa: E731
    f64 = lambda v: np.float64(np.float32(v))  # noqa: E731
    w = np.zeros(23333, np.float32)
    bi, bf, bg, bo_gate = 0.3, -0.7, 0.9, 1.1
    w[23040:23072] = bi
    w[23072:23104] = bf
    w[23104:23136] = bg
    w[23136:23168] = bo_gate
    w[23328:23333] = [0.0, 0.5, -0.5, 0.5, 0.25]  # ties between 1 and 3
    obs = np.ones(148)
    a, h, c, logits = oracle.lstm_step(w, obs, np.zeros(32), np.zeros(32))
    c_want = sig(f64(bi)) * np.tanh(f64(bg))
    h_want = sig(f64(bo_gate)) * np.tanh(c_want)
    np.testing.assert_allclose(c, c_want, rtol=1e-15)
    np.testing.assert_allclose(h, h_want, rtol=1e-15)
    assert a == 1  # lowest index among equal maxima
    # the forget gate scales an existing cell state
    _, _, c3, _ = oracle.lstm_step(w, obs, np.zeros(32), np.full(32, 2.0))
    np.testing.assert_allclose(c3, sig(f64(bf)) * 2.0 + c_want, rtol=1e-15)


def test_lstm_action_is_argmax_of_output_layer(oracle):
    w = np.zeros(23333, np.float32)
    for best in range(5):
        w[23328:23333] = 0.0
        w[23328 + best] = 1.0
        a, _, _, logits = oracle.lstm_step(w, np.zeros(148), np.zeros(32), np.zeros(32))
        assert a == best and logits[best] == pytest.approx(1.0)
