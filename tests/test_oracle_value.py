"""Pins for the oracle's value network (features, forward, loss gradient)."""
import math

import numpy as np
import pytest

import oracle
from statefmt import encode

NP = 855556
VH, VF = 512, 640
OFF_B1 = VH * VF
OFF_W2 = OFF_B1 + VH
OFF_B2 = OFF_W2 + VH * VH
OFF_W3 = OFF_B2 + VH
OFF_B3 = OFF_W3 + VH * VH
OFF_W4 = OFF_B3 + VH
OFF_B4 = OFF_W4 + 4 * VH


def test_layout():
    assert oracle.value_nparams() == NP == OFF_B4 + 4


def test_features_worked_example():
    # Player 0 to move holds 1, 6 (drawn this turn) and 14 (face up); player 1
    # holds 3, 10 (face up), 17.  Features written out by hand:
    #   part A (7 per tile: 4 owner seats relative to the mover, down/up, drawn)
    #     tile 1: seat 0, down -> 7, 11;   tile 6: seat 0, down, drawn -> 42, 46, 48
    #     tile 14: seat 0, up -> 98, 103;  tile 3: seat 1, down -> 22, 25
    #     tile 10: seat 1, up -> 71, 75;   tile 17: seat 1, down -> 120, 123
    #   part B (opponent 1, 13 values per slot, from 182):
    #     slot 0 (down, right neighbour 10): unknown tiles 0,2,3,4,5,7,8,9 -> values 0-4
    #     slot 1 (face-up 10): value 5 -> 200
    #     slot 2 (down, left neighbour 10): unknown tiles 11..13, 15..23 -> values 5-11
    s = encode([[1, 6, 14], [3, 10, 17]], {10, 14}, cur=0, drawn=6, ntiles=24)
    want = [7, 11, 42, 46, 48, 98, 103, 22, 25, 71, 75, 120, 123,
            182, 183, 184, 185, 186, 200] + list(range(182 + 26 + 5, 182 + 26 + 12))
    f = oracle.value_features(s)
    assert sorted(np.nonzero(f)[0].tolist()) == sorted(want)
    assert set(np.unique(f).tolist()) <= {0.0, 1.0}


def test_features_joker_and_seats():
    # 3 players, 26 tiles, mover is seat 2; seat 0 holds the white joker face
    # down, the black joker is in the pool -> every face-down slot may be a joker.
    s = encode([[25, 4], [0, 9], [12, 20]], set(), cur=2, drawn=20, ntiles=26)
    f = oracle.value_features(s)
    # tile 25 owned by seat 0 = relative seat 1, face down
    assert f[7 * 25 + 1] == 1 and f[7 * 25 + 4] == 1
    # tile 0 owned by seat 1 = relative seat 2
    assert f[7 * 0 + 2] == 1
    # opponent 1 (seat 0), slot 0 (the joker, face down): joker feasible
    assert f[182 + 12] == 1
    # opponent 2 (seat 1), slot 1 (tile 9, face down): values of unknown tiles
    base = 182 + (11 + 1) * 13
    unknown = [t for t in range(24) if t not in (12, 20)]
    assert sorted(np.nonzero(f[base:base + 12])[0].tolist()) == sorted({t // 2 for t in unknown})
    assert f[611:].sum() == 0


def _params(rng, scale=0.05):
    return (rng.standard_normal(NP) * scale).astype(np.float32)


def test_forward_closed_form_and_seat_mapping():
    # Zero weights everywhere except b3 and b4: every hidden unit of layer 3 is
    # GELU(b3), logits = W4 GELU(b3) + b4 with W4 = 0 -> logits = b4, so the
    # win probabilities are the softmax of b4 over the seats in play, mapped
    # from seats relative to the mover to absolute seats.
    p = np.zeros(NP, dtype=np.float32)
    p[OFF_B3:OFF_B3 + VH] = 0.7
    p[OFF_B4:OFF_B4 + 4] = [0.3, -1.2, 2.0, 5.0]
    s = encode([[1, 2], [3, 4], [5, 6]], set(), cur=1, drawn=None, ntiles=24)
    b4 = p[OFF_B4:OFF_B4 + 3].astype(np.float64)   # the stored float32 values
    e = np.exp(b4)
    soft = e / e.sum()
    got = oracle.value_forward(p, s)
    assert got[1] == pytest.approx(soft[0], rel=1e-12)   # relative seat 0 = the mover
    assert got[2] == pytest.approx(soft[1], rel=1e-12)
    assert got[0] == pytest.approx(soft[2], rel=1e-12)
    assert got[3] == 0.0
    # W4 row 0 = 1: logit 0 gains 512 * GELU(0.7), GELU in its tanh form,
    # which stays within 1e-3 of the exact 0.5 x (1 + erf(x / sqrt 2))
    p[OFF_W4:OFF_W4 + VH] = 1.0
    c = float(np.float32(0.7))
    g07 = 0.5 * c * (1 + math.tanh(math.sqrt(2 / math.pi) * (c + 0.044715 * c ** 3)))
    assert abs(g07 - 0.5 * c * (1 + math.erf(c / math.sqrt(2)))) < 1e-3
    z = b4 + np.array([VH * g07, 0.0, 0.0])
    e = np.exp(z - z.max())
    assert oracle.value_forward(p, s)[1] == pytest.approx(e[0] / e.sum(), rel=1e-9)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = _params(rng, 0.08)
    cfgs = [oracle.OracleConfig(nplayers=2, ntiles=24, deal=4, max_predraw=6),
            oracle.OracleConfig(nplayers=4, ntiles=26, deal=3, max_predraw=6, max_revealed=3)]
    states = np.concatenate([oracle.init_states(c, 4, 2) for c in cfgs])
    labels = rng.dirichlet(np.ones(4), size=len(states)).astype(np.float32)
    labels[:2, 2:] = 0
    labels[:2] /= labels[:2].sum(1, keepdims=True)
    loss, g = oracle.value_loss_grad(p, states, labels)
    assert np.isfinite(loss) and loss > 0
    h = 2.0 ** -10
    idx = list(rng.integers(0, NP, size=40)) + [OFF_B4, OFF_B4 + 3, OFF_W4 + 7, OFF_B1 + 5, OFF_B3 + 100]
    for i in idx:
        q = p.copy()
        q[i] = p[i] + h
        lp, _ = oracle.value_loss_grad(q, states, labels)
        q[i] = p[i] - h
        lm, _ = oracle.value_loss_grad(q, states, labels)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(g[i])) + 1e-7, (i, fd, g[i])


# ---- AdamW (Loshchilov and Hutter; Kingma and Ba) -------------------------

VH, VF = 512, 640
BIAS_RANGES = [(VH * VF, VH * VF + VH), (VH * VF + VH + VH * VH, VH * VF + 2 * VH + VH * VH),
               (VH * VF + 2 * VH + 2 * VH * VH, VH * VF + 3 * VH + 2 * VH * VH),
               (VH * VF + 3 * VH + 2 * VH * VH + 4 * VH, VH * VF + 3 * VH + 2 * VH * VH + 4 * VH + 4)]


def _is_bias():
    n = oracle.value_nparams()
    b = np.zeros(n, dtype=bool)
    for a, z in BIAS_RANGES:
        b[a:z] = True
    assert BIAS_RANGES[-1][1] == n
    return b


def test_adamw_first_step_is_sign_like():
    # From zero moments the bias corrections make mhat = g and vhat = g^2
    # exactly, so the step is g / (|g| + eps), plus wd * w on weight matrices.
    n = oracle.value_nparams()
    rng = np.random.default_rng(1)
    w0 = rng.normal(size=n)
    g = rng.normal(size=n) * 10.0 ** rng.integers(-6, 2, size=n)
    g[::97] = 0.0
    lr, wd, eps = 1e-3, 1e-4, 1e-8
    w, m, v = oracle.adamw_step(w0, np.zeros(n), np.zeros(n), g, 1, lr)
    dec = np.where(_is_bias(), 0.0, wd * w0)
    want = w0 - lr * (g / (np.abs(g) + eps) + dec)
    assert np.allclose(w, want, rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g, rtol=1e-15, atol=0) and np.allclose(v, 0.001 * g * g, rtol=1e-12, atol=0)
    # a zero gradient moves a matrix entry by decay alone and leaves a bias entry
    z = np.zeros(n)
    w1, _, _ = oracle.adamw_step(w0, z, z, z, 1, lr)
    bias = _is_bias()
    assert (w1[bias] == w0[bias]).all()
    assert np.allclose(w1[~bias], w0[~bias] * (1 - lr * wd), rtol=1e-15, atol=0)


def test_adamw_constant_gradient_closed_form():
    # A constant gradient keeps mhat = g and vhat = g^2 at every step (the
    # bias corrections undo the zero start), so with a = 1 - lr wd:
    #   w_k = a^k w_0 - lr s (1 - a^k) / (1 - a)   (matrices), w_0 - k lr s (biases),
    # s = g / (|g| + eps).
    n = oracle.value_nparams()
    rng = np.random.default_rng(2)
    w0 = rng.normal(size=n)
    g = rng.normal(size=n)
    lr, wd, eps, K = 1e-2, 1e-4, 1e-8, 25
    w, m, v = w0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, K + 1):
        w, m, v = oracle.adamw_step(w, m, v, g, t, lr)
    s = g / (np.abs(g) + eps)
    a = 1 - lr * wd
    want = np.where(_is_bias(), w0 - K * lr * s, a ** K * w0 - lr * s * (1 - a ** K) / (1 - a))
    assert np.allclose(w, want, rtol=0, atol=1e-11)
