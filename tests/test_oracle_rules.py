"""Pins for the oracle's game rules (Sec. II-A) and random playouts (Sec. II-B).

Checked against: rule invariants on traced playouts, the 88 root guesses of
Sec. III-A, the closed-form 1/k endgame, and exact win probabilities of tiny
endgames from the independent enumerator in bruteforce.py.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from bruteforce import exact_win_probs
from statefmt import decode, encode

CFG_2P = oracle.OracleConfig(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5)
CFG_3P = oracle.OracleConfig(nplayers=3, ntiles=24, deal=4, max_predraw=6, max_revealed=3)
CFG_4PJ = oracle.OracleConfig(nplayers=4, ntiles=26, deal=3, max_predraw=8, max_revealed=3)
CFGS = [CFG_2P, CFG_3P, CFG_4PJ]


def _check_state(d):
    T, P = d["T"], d["P"]
    seen = set()
    for h in d["hands"]:
        for t in h:
            assert 0 <= t < T
            assert t not in seen          # I1: a tile is in at most one hand
            seen.add(t)
        nums = [t for t in h if t < 24]
        assert nums == sorted(nums)       # I2: numbered tiles ascend (black before white)
    assert d["revealed"] <= seen          # face-up tiles are held by someone
    for p in range(P):
        hidden = [t for t in d["hands"][p] if t not in d["revealed"]]
        assert d["alive"][p] == (len(hidden) > 0)


def _next_alive(alive, c):
    p = c
    while True:
        p = (p + 1) % len(alive)
        if alive[p]:
            return p


def _check_transition(prev, d, cfg):
    """One guess (plus the draw that may follow) obeys Sec. II-A."""
    (t,) = tuple(d["revealed"] - prev["revealed"])
    c = prev["cur"]
    own = t in prev["hands"][c]
    if own:
        # wrong guess: the drawn tile turns face up, else the leftmost face-down one
        if prev["drawn"] is not None:
            assert t == prev["drawn"]
        else:
            assert t == next(u for u in prev["hands"][c] if u not in prev["revealed"])
    if d["winner"] is not None:
        return
    if own or d["cur"] != c:
        # the turn passed to the next player still in, who drew if the pool had tiles
        assert d["cur"] == _next_alive(d["alive"], c)
        held_before = sum(len(h) for h in prev["hands"])
        pool_before = cfg.ntiles - held_before
        n = d["cur"]
        if pool_before > 0:
            (new,) = tuple(set(d["hands"][n]) - set(prev["hands"][n]))
            assert d["drawn"] == new and new not in d["revealed"]
        else:
            assert d["drawn"] is None and d["hands"] == prev["hands"]
    else:
        # correct guess followed by another guess: same player, same drawn tile, no draw
        assert d["drawn"] == prev["drawn"] and d["hands"] == prev["hands"]
        assert cfg.cont_thr > 0


@pytest.mark.parametrize("cfg", CFGS, ids=["2p24", "3p24", "4p26j"])
def test_init_states_invariants(cfg):
    states = oracle.init_states(cfg, seed=11, n=64)
    deal_total = cfg.nplayers * cfg.deal
    for s in states:
        d = decode(s)
        _check_state(d)
        held = sum(len(h) for h in d["hands"])
        pool = cfg.ntiles - held
        assert held >= deal_total + 1 or pool == 0     # the root player has drawn
        assert held <= deal_total + cfg.max_predraw + 1
        assert d["winner"] is None
        for p in range(cfg.nplayers):
            assert len(d["revealed"] & set(d["hands"][p])) <= cfg.max_revealed
        if d["drawn"] is not None:
            assert d["drawn"] in d["hands"][d["cur"]] and d["drawn"] not in d["revealed"]


def test_init_states_deterministic_and_varied():
    a = oracle.init_states(CFG_2P, seed=5, n=32)
    b = oracle.init_states(CFG_2P, seed=5, n=32)
    c = oracle.init_states(CFG_2P, seed=6, n=32)
    assert (a == b).all()
    assert not (a == c).all()
    held = [sum(len(h) for h in decode(s)["hands"]) for s in a]
    assert len(set(held)) > 3   # histories of different lengths


@pytest.mark.parametrize("cfg", CFGS, ids=["2p24", "3p24", "4p26j"])
def test_playout_invariants(cfg):
    states = oracle.init_states(cfg, seed=3, n=24)
    for i, s in enumerate(states):
        for j in range(4):
            tr = oracle.playout_trace(cfg, s, seed=9, tree=i, j=j, leaf_id=0)
            prev = decode(s)
            assert 1 <= len(tr) <= cfg.ntiles      # I5: at most |T| guesses
            for k, st in enumerate(tr):
                d = decode(st)
                _check_state(d)
                assert prev["revealed"] <= d["revealed"]               # I3
                assert len(d["revealed"] - prev["revealed"]) == 1      # I4
                grew = [len(d["hands"][p]) - len(prev["hands"][p]) for p in range(cfg.nplayers)]
                assert all(g in (0, 1) for g in grew) and sum(grew) <= 1
                for p in range(cfg.nplayers):      # insertion keeps earlier tiles in order
                    old = prev["hands"][p]
                    assert [t for t in d["hands"][p] if t in old] == old
                _check_transition(prev, d, cfg)
                prev = d
            last = decode(tr[-1])
            assert last["winner"] is not None                          # I6
            assert [p for p in range(cfg.nplayers) if last["alive"][p]] == [last["winner"]]
            for st in tr[:-1]:
                assert decode(st)["winner"] is None


def _hands_pre_draw(T):
    # 2 players, 4 tiles each, all face down, player 0 to guess before drawing
    return encode([[0, 7, 12, 19], [2, 9, 14, 21]], set(), cur=0, drawn=None, ntiles=T)


def test_root_guess_count_matches_paper():
    # Sec. III-A: with position + number as the node key the root has 88
    # children (26 tiles, opponent holding four tiles): 4 slots x (26 - 4);
    # the value is read from the fixture that cites it
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_root_guesses.txt")
    rows = [list(map(int, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]
    for tiles, face_down, held, children in rows:
        assert face_down == 4 and held == 4
        assert oracle.legal_count(_hands_pre_draw(tiles)) == children
    assert oracle.legal_count(_hands_pre_draw(24)) == 80


@pytest.mark.parametrize("cfg", CFGS, ids=["2p24", "3p24", "4p26j"])
def test_legal_count_product_form(cfg):
    # I7: the legal set is (face-down slots of live opponents) x (identities
    # neither in the guesser's hand nor face up).
    for s in oracle.init_states(cfg, seed=21, n=48):
        d = decode(s)
        cur = d["cur"]
        slots = sum(len([t for t in d["hands"][q] if t not in d["revealed"]])
                    for q in range(cfg.nplayers) if q != cur and d["alive"][q])
        ids = cfg.ntiles - len(set(d["hands"][cur]) | d["revealed"])
        assert oracle.legal_count(s) == slots * ids


def _mc_close(cfg, state, exact, n=200000, seed=77):
    wins, _ = oracle.rollout(cfg, state, n, seed=seed, tree=1, leaf_id=2)
    assert wins.sum() == n
    for p, pr in exact.items():
        pr = float(pr)
        sd = math.sqrt(max(pr * (1 - pr), 1e-12) / n)
        assert abs(wins[p] / n - pr) <= 5 * sd + 1e-9, (p, wins[p] / n, pr)
    for p in range(4):
        if p not in exact:
            assert wins[p] == 0


@pytest.mark.parametrize("k", [2, 3, 5])
def test_closed_form_one_over_k(k):
    # Player 0's only face-down tile is the one it drew; player 1 has one
    # face-down tile whose slot is unconstrained; k-1 tiles remain in the pool.
    # A correct guess (prob 1/k) eliminates player 1, a wrong one eliminates
    # player 0, so player 0 wins with probability exactly 1/k.
    pool = list(range(24 - (k - 1), 24))
    rest = [t for t in range(24) if t not in pool]
    h1 = [rest[0]] + rest[1:12]          # face-down tile first
    h0 = rest[12:]
    drawn = h0[-1]
    revealed = set(h0[:-1]) | set(h1[1:])
    s = encode([h0, h1], revealed, cur=0, drawn=drawn, ntiles=24)
    exact = exact_win_probs([h0, h1], revealed, 0, drawn, 24, 0)
    assert exact[0] == Fraction(1, k)
    cfg = oracle.OracleConfig(cont_thr=1 << 31)
    _mc_close(cfg, s, {0: 1 / k, 1: 1 - 1 / k})


ENDGAMES = {
    # 2 players, 24 tiles, five tiles in the pool, two face-down tiles each
    "2p_pool5": dict(hands=[[0, 2, 4, 6, 8, 10, 12, 14, 16], [1, 3, 5, 7, 9, 11, 13, 15, 17, 19]],
                     hidden={0, 16, 1, 5}, cur=0, drawn=16, T=24),
    # 3 players, 26 tiles, the black joker in the pool, the white one face down
    "3p_joker": dict(hands=[[0, 1, 2, 3, 4, 5, 6, 7], [8, 9, 10, 11, 12, 13, 14, 15],
                            [16, 17, 18, 19, 20, 21, 22, 23, 25]],
                     hidden={7, 9, 18, 25}, cur=0, drawn=7, T=26),
    # 4 players, 24 tiles, empty pool, one player already out
    "4p_out": dict(hands=[[0, 1, 2, 3, 4, 5], [6, 7, 8, 9, 10, 11], [12, 13, 14, 15, 16, 17],
                          [18, 19, 20, 21, 22, 23]],
                   hidden={2, 5, 7, 8, 23, 21}, cur=1, drawn=None, T=24),
}


@pytest.mark.parametrize("name", sorted(ENDGAMES))
@pytest.mark.parametrize("cont", [0, 1 << 31])
def test_tiny_endgames_exact(name, cont):
    e = ENDGAMES[name]
    held = {t for h in e["hands"] for t in h}
    revealed = held - e["hidden"]
    exact = exact_win_probs(e["hands"], revealed, e["cur"], e["drawn"], e["T"], cont / 2 ** 32)
    assert sum(exact.values()) == 1
    P = len(e["hands"])
    s = encode(e["hands"], revealed, cur=e["cur"], drawn=e["drawn"], ntiles=e["T"])
    cfg = oracle.OracleConfig(nplayers=P, ntiles=e["T"], cont_thr=cont)
    _mc_close(cfg, s, exact)


def test_playout_words_counted():
    s = oracle.init_states(CFG_2P, seed=1, n=1)[0]
    _, words = oracle.rollout(CFG_2P, s, 64, seed=3, tree=0, leaf_id=0)
    assert 64 * 10 < words < 64 * 200
