"""Pins of the oracle's paper controller (App. B.5) and its world wiring.

* parameter count: the architecture built from torch layers (conv 3x3/2,
  average pool 2x2/1, conv 3x3/2, pool, LSTM(4) with one bias per gate,
  dense 8, dense 5) has the 2445 parameters the paper states;
* forward pass: torch conv2d / avg_pool2d / LSTMCell / linear in float64
  with the same weights;
* view: padded numpy slices of the three channels;
* sampling: closed forms (uniform and one-hot distributions), empirical
  frequencies against the softmax at temperature 1/50, the action uniform
  against the tests' own numpy Philox;
* world: the previous-action and ate inputs, mutation of exactly the 2445
  parameters, the paper preset's invariants.
"""
import numpy as np
import pytest
import torch

from paper_2302_09334_gb300.params import EcoParams, paper_natural
from tests.philox_np import philox

PAPER_PARAM_COUNT = 2445        # App. B.5: "only 2445 parameters"


class TorchPaperNet(torch.nn.Module):
    def __init__(self):
        super().__init__()
        self.c1 = torch.nn.Conv2d(3, 4, 3, stride=2, padding=1)
        self.c2 = torch.nn.Conv2d(4, 8, 3, stride=2, padding=1)
        self.lstm = torch.nn.LSTMCell(78, 4, bias=True)
        self.d1 = torch.nn.Linear(82, 8)
        self.d2 = torch.nn.Linear(8, 5)

    def embed(self, obs_hwc):
        x = torch.as_tensor(obs_hwc).permute(2, 0, 1)[None]          # NCHW
        x = torch.nn.functional.avg_pool2d(self.c1(x), 2, stride=1)
        x = torch.nn.functional.avg_pool2d(self.c2(x), 2, stride=1)   # [1, 8, 3, 3]
        return x[0].permute(1, 2, 0).reshape(-1)                       # [y][x][c]


def _load(net, w, oracle):
    o = oracle.PC_OFF
    t = lambda a, b, shape: torch.tensor(w[a:b].reshape(shape), dtype=torch.float64)  # noqa
    with torch.no_grad():
        net.c1.weight.copy_(t(o["W1"], o["B1"], (4, 3, 3, 3)).permute(0, 3, 1, 2))
        net.c1.bias.copy_(t(o["B1"], o["W2"], (4,)))
        net.c2.weight.copy_(t(o["W2"], o["B2"], (8, 3, 3, 4)).permute(0, 3, 1, 2))
        net.c2.bias.copy_(t(o["B2"], o["WI"], (8,)))
        net.lstm.weight_ih.copy_(t(o["WI"], o["WH"], (16, 78)))
        net.lstm.weight_hh.copy_(t(o["WH"], o["BL"], (16, 4)))
        net.lstm.bias_ih.copy_(t(o["BL"], o["D1"], (16,)))
        net.lstm.bias_hh.zero_()
        net.d1.weight.copy_(t(o["D1"], o["DB1"], (8, 82)))
        net.d1.bias.copy_(t(o["DB1"], o["D2"], (8,)))
        net.d2.weight.copy_(t(o["D2"], o["DB2"], (5, 8)))
        net.d2.bias.copy_(t(o["DB2"], 2445, (5,)))


def test_parameter_count_is_the_papers(oracle):
    net = TorchPaperNet()
    n = sum(p.numel() for p in net.parameters())
    # torch keeps two LSTM bias vectors; the paper's count has one per gate
    assert n - net.lstm.bias_hh.numel() == PAPER_PARAM_COUNT
    assert oracle.param_count(oracle.CTRL_PAPER) == PAPER_PARAM_COUNT == oracle.PC_NPARAM
    assert oracle.param_count(oracle.CTRL_LSTM32) == 23333
    assert oracle.param_count(7) == -1
    offs = sorted(oracle.PC_OFF.values()) + [2445]
    sizes = np.diff(offs)
    assert list(sizes) == [108, 4, 288, 8, 1248, 64, 16, 656, 8, 40, 5]
    # the CNN maps the 15x15 view to 3x3x8 = 72 features
    assert net.embed(np.zeros((15, 15, 3), np.float32)).numel() == 72


def test_forward_matches_torch(oracle):
    rng = np.random.default_rng(11)
    net = TorchPaperNet().double()
    for trial in range(6):
        w = (rng.standard_normal(2445) * 0.3).astype(np.float32)
        _load(net, w, oracle)
        obs = rng.integers(0, 2, (15, 15, 3)).astype(np.float64)
        prev, ate = int(rng.integers(0, 5)), int(rng.integers(0, 2))
        h = rng.uniform(-1, 1, 4)
        c = rng.uniform(-2, 2, 4)
        h2, c2, logits = oracle.pc_forward(w, obs, prev, ate, h, c)
        with torch.no_grad():
            emb = torch.cat([net.embed(obs), torch.nn.functional.one_hot(
                torch.tensor(prev), 5).double(), torch.tensor([float(ate)], dtype=torch.float64)])
            th, tc = net.lstm(emb[None], (torch.tensor(h)[None], torch.tensor(c)[None]))
            d = torch.tanh(net.d1(torch.cat([emb, th[0]])))
            tl = net.d2(d)
        np.testing.assert_allclose(h2, th[0].numpy(), rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(c2, tc[0].numpy(), rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(logits, tl.numpy(), rtol=1e-12, atol=1e-13)


def test_view_matches_slicing(oracle):
    rng = np.random.default_rng(5)
    p = EcoParams(H=23, W=31, controller=1)
    res = (rng.random((p.H, p.W)) < 0.4).astype(np.uint8)
    wall = (rng.random((p.H, p.W)) < 0.2).astype(np.uint8)
    slot_map = np.where(rng.random((p.H, p.W)) < 0.3, 1, -1).astype(np.int32)
    r = np.pad(res, 7)
    a = np.pad((slot_map >= 0).astype(np.uint8), 7)
    wl = np.pad(wall, 7, constant_values=1)
    for (y, x) in [(0, 0), (22, 30), (11, 15), (3, 27), (20, 2)]:
        got = oracle.pc_observe(p.asdict(), res, wall, slot_map, y, x)
        want = np.stack([r[y:y + 15, x:x + 15], a[y:y + 15, x:x + 15],
                         wl[y:y + 15, x:x + 15]], axis=-1).astype(np.float64)
        want[7, 7, 1] = 0.0
        np.testing.assert_array_equal(got, want)


def test_sampling_closed_forms(oracle):
    flat = np.zeros(5)
    for u in np.linspace(0, 0.999, 37):
        assert oracle.pc_sample(flat, u) == min(int(u / 0.2 + 1e-12), 4)
    for k in range(5):
        lg = np.zeros(5)
        lg[k] = 1.0                  # 50x the logit gap: probability 1 - 4e-22
        for u in (1e-6, 0.3, 0.999999):
            assert oracle.pc_sample(lg, u) == k
        # u = 0 lies below every cumulative probability: action 0
        assert oracle.pc_sample(lg, 0.0) == 0
    # two tied leaders share the mass equally
    lg = np.array([0.0, 0.5, 0.5, 0.0, -1.0])
    assert oracle.pc_sample(lg, 0.49) == 1 and oracle.pc_sample(lg, 0.51) == 2


def test_sampling_frequencies(oracle):
    rng = np.random.default_rng(6)
    lg = np.array([0.01, 0.03, -0.02, 0.0, 0.025])
    z = np.exp(50 * (lg - lg.max()))
    prob = z / z.sum()
    n = 40000
    us = rng.random(n)
    counts = np.bincount([oracle.pc_sample(lg, u) for u in us], minlength=5)
    bound = 5 * np.sqrt(prob * (1 - prob) / n)
    assert np.all(np.abs(counts / n - prob) < bound)


def test_action_uniform_is_philox_word(oracle):
    seed = 0x123456789A
    for t, s in [(0, 0), (5, 17), (1000, 4095)]:
        word = philox(s, t, oracle.TAG_ACT, 0, seed & 0xFFFFFFFF, seed >> 32)[0]
        assert oracle.action_uniform(seed, t, s) == (int(word) >> 8) / 2**24


def _quiet_paper(**kw):
    base = dict(H=12, W=20, capacity=64, n_agents0=10, p_class=(0.0, 0.0, 0.0, 0.0),
                p_spont=0.0, e_decay=0.0, t_repr=2**31 - 1, wall_kills=0, controller=1)
    base.update(kw)
    return EcoParams(**base)


def test_world_inputs_and_mutation(oracle):
    p = _quiet_paper(res_init_p=0.3, t_repr=6, e_repr=0.5)
    ow = oracle.OracleWorld(p.asdict(), 3)
    assert np.all(ow.weights[:p.n_agents0, 2445:] == 0)       # only 2445 parameters drawn
    w0 = oracle.fill_normals_n(3, oracle.TAG_INIT_W, 0, 2, p.w_init_std, 2445)
    np.testing.assert_array_equal(ow.weights[2, :2445], w0)
    births = checked = 0
    for step in range(20):
        live = ow.alive.astype(bool).copy()
        prev, ate = ow.prev_action.copy(), ow.ate.copy()
        h, c = ow.h.copy(), ow.c.copy()
        y, x = ow.y.copy(), ow.x.copy()
        res, slot_map = ow.res.copy(), ow.slot_map.copy()   # regrowth is off
        weights = ow.weights.copy()
        t = ow.t
        ow.step()
        nb = int(ow.counters[oracle.C_BIRTHS_LAST])
        reborn = set(int(v) for v in ow.birth_child[:nb])
        # each acting agent's controller saw the start-of-step view, its
        # previous move and its ate bit, and sampled with its own uniform
        for s in np.flatnonzero(live):
            if s in reborn:
                continue
            obs = oracle.pc_observe(p.asdict(), res, ow.wall, slot_map, y[s], x[s])
            h2, c2, lg = oracle.pc_forward(weights[s], obs, prev[s], ate[s], h[s], c[s])
            np.testing.assert_array_equal(ow.h[s, :4], h2)
            np.testing.assert_array_equal(ow.c[s, :4], c2)
            np.testing.assert_array_equal(ow.logits[s], lg)
            assert ow.action[s] == oracle.pc_sample(lg, oracle.action_uniform(3, t, s))
            checked += 1
        for k in range(nb):
            par, ch = int(ow.birth_parent[k]), int(ow.birth_child[k])
            want = oracle.fill_normals_n(3, oracle.TAG_MUT, t, par, p.mut_std, 2445,
                                         base=weights[par, :2445])
            np.testing.assert_array_equal(ow.weights[ch, :2445], want)
            assert np.all(ow.weights[ch, 2445:] == 0)
            assert ow.prev_action[ch] == 0 and ow.ate[ch] == 0
        births += nb
        moved = live & ow.alive.astype(bool)
        moved[list(reborn)] = False
        np.testing.assert_array_equal(ow.prev_action[moved], ow.move_action[moved])
        assert set(np.unique(ow.ate[~ow.alive.astype(bool)])) <= {0}
    assert births > 0 and checked > 100
    assert (ow.prev_action[ow.alive.astype(bool)] > 0).any()


def test_paper_preset_runs_with_invariants(oracle):
    p = paper_natural()
    assert p.controller == 1 and p.capacity == 1000 and p.n_agents0 == 330
    ow = oracle.OracleWorld(p.asdict(), 0)
    pop = ow.population
    res0 = int(ow.res.sum())
    assert 14000 < res0 < 18000                 # ~16,000 initial resources
    for _ in range(15):
        ow.step()
        c = ow.counters
        assert ow.population == pop + c[oracle.C_BIRTHS_LAST] - c[oracle.C_DEATHS_LAST]
        pop = ow.population
        alive = np.flatnonzero(ow.alive)
        cells = ow.y[alive] * p.W + ow.x[alive]
        assert len(np.unique(cells)) == pop and not ow.wall.ravel()[cells].any()
        assert np.all(ow.energy[alive] <= np.float32(3.0))
        assert set(np.unique(ow.action[alive])) <= set(range(5))
