"""Pins of the oracle's error magnitudes (or_lstm_mag, or_pc_mag), the
per-element scale of the RNN parity tolerance.

E is a running error analysis: the magnitude by which an evaluation whose
every operation rounds with relative error at most eps can differ from the
exact outputs, to first order, is eps * E.  Two independent checks:

  * first-order worst case by automatic differentiation: the same forward
    pass written with torch ops, with a rounding error injected at every
    operation (a dot product's result off by up to eps (|b| + sum |w v|),
    any other result off by up to eps |result|, an input h or c off by up
    to eps times its given magnitude); the worst case over all choices of
    those errors is B = sum over operations of |d output / d error| times
    the operation's bound, computed from the Jacobian.  E must be at least
    B for every output (a dropped term or a wrong derivative makes it
    smaller somewhere), and not far above it (triangle inequality over the
    paths only);
  * simulated low-precision arithmetic: the LSTM step evaluated with every
    product, sum and activation rounded to a 20-bit mantissa (stochastic
    rounding, sequential sums) stays within (n + 2) 2^-20 E of the FP64
    result for every output, n = 180 the longest dot product.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as orc


def _lstm_case(rng, std):
    w = rng.normal(0.0, std, orc.NPARAM).astype(np.float32)
    obs = (rng.random(orc.NOBS) < 0.3).astype(np.float64)
    obs[147] = rng.uniform(0.0, 3.0)
    h = rng.uniform(-1.0, 1.0, orc.HID)
    c = rng.uniform(-3.0, 3.0, orc.HID)
    eh = rng.uniform(0.0, 5.0, orc.HID)
    ec = rng.uniform(0.0, 5.0, orc.HID)
    return w, obs, h, c, eh, ec


def _lstm_worst_case(w, obs, h, c, eh, ec):
    """B for (h', c', logits) of one LSTM step: first-order worst case over
    the rounding errors of every operation (torch autograd, float64)."""
    W = torch.tensor(w, dtype=torch.float64)
    Wx = W[:orc.OFF_B].view(4 * orc.HID, orc.NOBS + orc.HID)
    b = W[orc.OFF_B:orc.OFF_WO]
    Wo = W[orc.OFF_WO:orc.OFF_BO].view(orc.NACT, orc.HID)
    bo = W[orc.OFF_BO:orc.NPARAM]
    obs_t, h_t, c_t = (torch.tensor(a, dtype=torch.float64) for a in (obs, h, c))
    eh_t, ec_t = torch.tensor(eh), torch.tensor(ec)
    H = orc.HID
    sizes = {"h": H, "c": H, "z": 4 * H, "i": H, "f": H, "g": H, "o": H, "fc": H, "ig": H,
             "cn": H, "tc": H, "hn": H, "l": orc.NACT}
    scale = {}

    def forward(flat, record=False):
        d, k = {}, 0
        for name, n in sizes.items():
            d[name] = flat[k:k + n]
            k += n

        def rnd(name, value, bound):
            if record:
                scale[name] = bound.detach().abs()
            return value + d[name] * scale[name]

        hin = h_t + d["h"] * eh_t
        cin = c_t + d["c"] * ec_t
        v = torch.cat([obs_t, hin])
        z = rnd("z", Wx @ v + b, b.abs() + Wx.abs() @ v.abs())
        gi = rnd("i", torch.sigmoid(z[0:H]), torch.sigmoid(z[0:H]))
        gf = rnd("f", torch.sigmoid(z[H:2 * H]), torch.sigmoid(z[H:2 * H]))
        gg = rnd("g", torch.tanh(z[2 * H:3 * H]), torch.tanh(z[2 * H:3 * H]))
        go = rnd("o", torch.sigmoid(z[3 * H:]), torch.sigmoid(z[3 * H:]))
        fc = rnd("fc", gf * cin, gf * cin)
        ig = rnd("ig", gi * gg, gi * gg)
        cn = rnd("cn", fc + ig, fc + ig)
        tc = rnd("tc", torch.tanh(cn), torch.tanh(cn))
        hn = rnd("hn", go * tc, go * tc)
        lg = rnd("l", Wo @ hn + bo, bo.abs() + Wo.abs() @ hn.abs())
        return torch.cat([hn, cn, lg])

    n = sum(sizes.values())
    zero = torch.zeros(n, dtype=torch.float64)
    forward(zero, record=True)
    J = torch.autograd.functional.jacobian(forward, zero)
    B = J.abs().sum(dim=1).numpy()
    return B[:H], B[H:2 * H], B[2 * H:]


@pytest.mark.parametrize("std", [0.1, 0.5, 1.0])
def test_lstm_magnitude_bounds_first_order_worst_case(std):
    rng = np.random.default_rng(7)
    ratios = []
    for _ in range(12):
        w, obs, h, c, eh, ec = _lstm_case(rng, std)
        Eh, Ec, El = orc.lstm_mag(w, obs, h, c, eh, ec)
        Bh, Bc, Bl = _lstm_worst_case(w, obs, h, c, eh, ec)
        for E, B, what in ((Eh, Bh, "h"), (Ec, Bc, "c"), (El, Bl, "logits")):
            assert (B <= E * (1 + 1e-12) + 1e-300).all(), (what, (B / E).max())
            ratios.append(E / B)
    r = np.concatenate(ratios)
    # E follows every path with |derivatives|; only cancellation between
    # paths (of h's magnitude through the four gates) can make it larger
    assert np.median(r) < 1.5 and r.max() < 20.0, (np.median(r), r.max())


def test_lstm_magnitude_exact_inputs_and_bias_only():
    """With zero weights the gates are the biases' logistic / tanh values:
    E follows from the rules by hand for one unit."""
    w = np.zeros(orc.NPARAM, np.float32)
    b = np.array([0.3, -0.7, 0.9, 0.2], np.float32)          # i, f, g, o of unit 5
    for gate in range(4):
        w[orc.OFF_B + gate * orc.HID + 5] = b[gate]
    w[orc.OFF_WO + 2 * orc.HID + 5] = np.float32(-1.5)       # logit 2 reads unit 5
    w[orc.OFF_BO + 2] = np.float32(0.25)
    obs = np.zeros(orc.NOBS)
    h = np.zeros(orc.HID)
    c = np.zeros(orc.HID)
    c[5] = 0.8
    Eh, Ec, El = orc.lstm_mag(w, obs, h, c)
    s = lambda x: 1 / (1 + np.exp(-float(x)))
    bi, bf, bg, bo_ = (float(x) for x in b)
    gi, gf, gg, go = s(bi), s(bf), np.tanh(bg), s(bo_)
    Ei = gi * (1 - gi) * abs(bi) + gi
    Ef = gf * (1 - gf) * abs(bf) + gf
    Eg = (1 - gg * gg) * abs(bg) + abs(gg)
    Eo = go * (1 - go) * abs(bo_) + go
    cn = gf * 0.8 + gi * gg
    Ecn = (0.8 * Ef + gf * 0.8) + (gi * Eg + abs(gg) * Ei + abs(gi * gg)) + abs(cn)
    tc = np.tanh(cn)
    hn = go * tc
    Ehn = go * ((1 - tc * tc) * Ecn + abs(tc)) + abs(tc) * Eo + abs(hn)
    assert Ec[5] == pytest.approx(Ecn, rel=1e-12)
    assert Eh[5] == pytest.approx(Ehn, rel=1e-12)
    assert El[2] == pytest.approx(0.25 + 1.5 * (abs(hn) + Ehn), rel=1e-12)
    # the other units: zero pre-activations, zero cell state
    other = [j for j in range(orc.HID) if j != 5]
    e0 = 0.5 * 0.0 + 0.5                                    # a gate at z = 0
    assert Ec[other] == pytest.approx(0.0 + (0.5 * 0.0 + 0.0 * e0 + 0.0))
    assert El[[0, 1, 3, 4]] == pytest.approx(0.0)


def _round_mantissa(x, bits, rng):
    """x rounded to `bits` mantissa bits, stochastically (unbiased)."""
    m, e = np.frexp(np.asarray(x, np.float64))
    scaled = m * (1 << bits)
    lo = np.floor(scaled)
    up = rng.random(np.shape(scaled)) < (scaled - lo)
    return np.ldexp((lo + up) / (1 << bits), e)


def _lstm_low_precision(w, obs, h, c, bits, rng):
    r = lambda x: _round_mantissa(x, bits, rng)
    H = orc.HID
    W = w.astype(np.float64)
    Wx = W[:orc.OFF_B].reshape(4 * H, orc.NOBS + H)
    v = np.concatenate([obs, h])
    acc = W[orc.OFF_B:orc.OFF_WO].copy()
    for k in range(v.size):                       # sequential sums, rounded every op
        acc = r(acc + r(Wx[:, k] * v[k]))
    sig = lambda z: r(1.0 / (1.0 + np.exp(-z)))
    gi, gf, gg, go = sig(acc[:H]), sig(acc[H:2 * H]), r(np.tanh(acc[2 * H:3 * H])), \
        sig(acc[3 * H:])
    cn = r(r(gf * c) + r(gi * gg))
    hn = r(go * r(np.tanh(cn)))
    Wo = W[orc.OFF_WO:orc.OFF_BO].reshape(orc.NACT, H)
    lg = W[orc.OFF_BO:orc.NPARAM].copy()
    for j in range(H):
        lg = r(lg + r(Wo[:, j] * hn[j]))
    return hn, cn, lg


@pytest.mark.parametrize("std", [0.1, 0.5])
def test_lstm_magnitude_covers_low_precision_evaluations(std):
    rng = np.random.default_rng(11)
    bits = 20
    eps = (orc.NOBS + orc.HID + 2) * 2.0 ** -bits
    worst = 0.0
    for _ in range(10):
        w, obs, h, c, _, _ = _lstm_case(rng, std)
        Eh, Ec, El = orc.lstm_mag(w, obs, h, c)
        ah, ac, alg = orc.lstm_step(w, obs, h, c)[1:]
        for trial in range(3):
            lh, lc, llg = _lstm_low_precision(w, obs, h, c, bits, rng)
            for got, ref, E in ((lh, ah, Eh), (lc, ac, Ec), (llg, alg, El)):
                err = np.abs(got - ref)
                assert (err <= eps * E).all(), (err / (eps * E)).max()
                worst = max(worst, float((err / (eps * E)).max()))
    assert worst > 1e-3   # the bound is not vacuous


def _pc_case(rng, std):
    w = rng.normal(0.0, std, orc.PC_NPARAM).astype(np.float32)
    obs = (rng.random((orc.PC_VIEW, orc.PC_VIEW, 3)) < 0.25).astype(np.float64)
    prev = int(rng.integers(0, orc.NACT))
    ate = int(rng.integers(0, 2))
    h = rng.uniform(-1.0, 1.0, orc.PC_HID)
    c = rng.uniform(-3.0, 3.0, orc.PC_HID)
    eh = rng.uniform(0.0, 5.0, orc.PC_HID)
    ec = rng.uniform(0.0, 5.0, orc.PC_HID)
    return w, obs, prev, ate, h, c, eh, ec


def _pc_worst_case(w, obs, prev, ate, h, c, eh, ec):
    """B for (h', c', logits) of one paper-controller step, as for the LSTM:
    torch conv2d / avg_pool2d / LSTM cell / dense layers in float64 with an
    injected rounding error at every operation."""
    import torch.nn.functional as F
    W = torch.tensor(w, dtype=torch.float64)
    P = orc.PC_OFF
    w1 = W[P["W1"]:P["B1"]].view(4, 3, 3, 3).permute(0, 3, 1, 2)
    b1 = W[P["B1"]:P["W2"]]
    w2 = W[P["W2"]:P["B2"]].view(8, 3, 3, 4).permute(0, 3, 1, 2)
    b2 = W[P["B2"]:P["WI"]]
    wi = W[P["WI"]:P["WH"]].view(16, 78)
    wh = W[P["WH"]:P["BL"]].view(16, 4)
    bl = W[P["BL"]:P["D1"]]
    d1 = W[P["D1"]:P["DB1"]].view(8, 82)
    db1 = W[P["DB1"]:P["D2"]]
    d2 = W[P["D2"]:P["DB2"]].view(5, 8)
    db2 = W[P["DB2"]:orc.PC_NPARAM]
    x = torch.tensor(obs, dtype=torch.float64).permute(2, 0, 1)[None]
    onehot = torch.zeros(5, dtype=torch.float64)
    onehot[prev] = 1.0
    tail = torch.cat([onehot, torch.tensor([float(ate)], dtype=torch.float64)])
    h_t, c_t = torch.tensor(h), torch.tensor(c)
    eh_t, ec_t = torch.tensor(eh), torch.tensor(ec)
    sizes = {"h": 4, "c": 4, "a1": 256, "p1": 196, "a2": 128, "p2": 72, "z": 16, "i": 4,
             "f": 4, "g": 4, "o": 4, "fc": 4, "ig": 4, "cn": 4, "tc": 4, "hn": 4, "dz": 8,
             "d": 8, "l": 5}
    scale = {}

    def forward(flat, record=False):
        d, k = {}, 0
        for name, n in sizes.items():
            d[name] = flat[k:k + n]
            k += n

        def rnd(name, value, bound):
            if record:
                scale[name] = bound.detach().abs().reshape(-1)
            return value + (d[name] * scale[name]).reshape(value.shape)

        hin = h_t + d["h"] * eh_t
        cin = c_t + d["c"] * ec_t
        a1 = rnd("a1", F.conv2d(x, w1, b1, stride=2, padding=1),
                 F.conv2d(x.abs(), w1.abs(), b1.abs(), stride=2, padding=1))
        p1 = F.avg_pool2d(a1, 2, stride=1)
        p1 = rnd("p1", p1, p1)
        a2 = rnd("a2", F.conv2d(p1, w2, b2, stride=2, padding=1),
                 F.conv2d(p1.abs(), w2.abs(), b2.abs(), stride=2, padding=1))
        p2 = F.avg_pool2d(a2, 2, stride=1)
        p2 = rnd("p2", p2, p2)
        emb = torch.cat([p2[0].permute(1, 2, 0).reshape(72), tail])
        z = rnd("z", wi @ emb + wh @ hin + bl, bl.abs() + wi.abs() @ emb.abs() +
                wh.abs() @ hin.abs())
        gi = rnd("i", torch.sigmoid(z[0:4]), torch.sigmoid(z[0:4]))
        gf = rnd("f", torch.sigmoid(z[4:8]), torch.sigmoid(z[4:8]))
        gg = rnd("g", torch.tanh(z[8:12]), torch.tanh(z[8:12]))
        go = rnd("o", torch.sigmoid(z[12:16]), torch.sigmoid(z[12:16]))
        fc = rnd("fc", gf * cin, gf * cin)
        ig = rnd("ig", gi * gg, gi * gg)
        cn = rnd("cn", fc + ig, fc + ig)
        tc = rnd("tc", torch.tanh(cn), torch.tanh(cn))
        hn = rnd("hn", go * tc, go * tc)
        u = torch.cat([emb, hn])
        dz = rnd("dz", d1 @ u + db1, db1.abs() + d1.abs() @ u.abs())
        dd = rnd("d", torch.tanh(dz), torch.tanh(dz))
        lg = rnd("l", d2 @ dd + db2, db2.abs() + d2.abs() @ dd.abs())
        return torch.cat([hn, cn, lg])

    n = sum(sizes.values())
    zero = torch.zeros(n, dtype=torch.float64)
    forward(zero, record=True)
    J = torch.autograd.functional.jacobian(forward, zero)
    B = J.abs().sum(dim=1).numpy()
    return B[:4], B[4:8], B[8:]


@pytest.mark.parametrize("std", [0.1, 0.5])
def test_paper_controller_magnitude_bounds_first_order_worst_case(std):
    rng = np.random.default_rng(5)
    ratios = []
    for _ in range(10):
        w, obs, prev, ate, h, c, eh, ec = _pc_case(rng, std)
        Eh, Ec, El = orc.pc_mag(w, obs, prev, ate, h, c, eh, ec)
        # the magnitudes belong to the oracle's own forward pass
        fh, fc_, _ = orc.pc_forward(w, obs, prev, ate, h, c)
        Bh, Bc, Bl = _pc_worst_case(w, obs, prev, ate, h, c, eh, ec)
        for E, B, what in ((Eh, Bh, "h"), (Ec, Bc, "c"), (El, Bl, "logits")):
            assert (B <= E * (1 + 1e-12) + 1e-300).all(), (what, (B / E).max())
            ratios.append(E / B)
        assert np.isfinite(fh).all() and np.isfinite(fc_).all()
    r = np.concatenate(ratios)
    # the convolutions' and pools' overlapping windows give many paths per
    # output, whose signs cancel in B but not in E
    assert np.median(r) < 5.0 and r.max() < 50.0, (np.median(r), r.max())


def test_world_keeps_magnitudes_per_slot():
    """The world's stored magnitudes are or_lstm_mag of each agent's step,
    from the previous step's magnitudes (recomputed here from the agent's
    inputs: regrown plane, start-of-step occupancy, energy, h, c); a
    newborn's start at zero; sync (state written from outside) zeroes them."""
    from paper_2302_09334_gb300.params import small_20x40
    p = small_20x40().replace(t_repr=3, e_decay=0.0)
    ow = orc.OracleWorld(p.asdict(), 3)
    ow.step()
    for _ in range(3):
        t = ow.t
        before = {k: getattr(ow, k).copy() for k in
                  ("res", "wall", "slot_map", "y", "x", "energy", "h", "c", "mag_h", "mag_c",
                   "alive")}
        ow.step()
        res_new = orc.regrow(p.asdict(), 3, t, before["res"], before["wall"])
        for s in np.flatnonzero(before["alive"])[:6]:
            obs = orc.observe(p.asdict(), res_new, before["wall"], before["slot_map"],
                              before["y"][s], before["x"][s], before["energy"][s])
            Eh, Ec, El = orc.lstm_mag(ow.weights[s], obs, before["h"][s], before["c"][s],
                                      before["mag_h"][s], before["mag_c"][s])
            np.testing.assert_array_equal(ow.mag_h[s], Eh)
            np.testing.assert_array_equal(ow.mag_c[s], Ec)
            np.testing.assert_array_equal(ow.mag_logits[s], El)
        nb = int(ow.counters[orc.C_BIRTHS_LAST])
        for ch in ow.birth_child[:nb]:
            assert not ow.mag_h[ch].any() and not ow.mag_c[ch].any()
    assert ow.counters[orc.C_BIRTHS] > 0
    ow.sync()
    assert not ow.mag_h.any() and not ow.mag_c.any() and not ow.mag_logits.any()


def test_magnitude_tracking_leaves_the_step_unchanged():
    """The magnitudes are test support: a world stepped without them has
    exactly the same state."""
    from paper_2302_09334_gb300.params import small_20x40
    p = small_20x40().replace(t_repr=5)
    a = orc.OracleWorld(p.asdict(), 5)
    b = orc.OracleWorld(p.asdict(), 5, magnitudes=False)
    for _ in range(30):
        a.step()
        b.step()
    for f in ("res", "slot_map", "alive", "y", "x", "energy", "h", "c", "logits", "weights",
              "counters", "action"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)
    assert a.counters[orc.C_BIRTHS] > 0
    assert not b.mag_h.any() and a.mag_h[a.alive.astype(bool)].any()
