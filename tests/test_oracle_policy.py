"""Pins for the oracle's ordering-aware playout policy: identities restricted
to those that fit between a face-down slot's nearest face-up numbered
neighbours in the opponent's sorted row (jokers anywhere)."""
import numpy as np
import pytest

import oracle
from bruteforce import exact_win_probs
from statefmt import decode, encode
from test_oracle_rules import ENDGAMES, _mc_close


def _codes(q, s, xs):
    return [(q << 10) | (s << 5) | x for x in xs]


def test_kept_guesses_written_out():
    # mover 0 holds 1, 6 (drawn), 14 (face up); opponent 1 holds 3, 10 (face up), 17
    s = encode([[1, 6, 14], [3, 10, 17]], {10, 14}, cur=0, drawn=6, ntiles=24)
    unknown = [x for x in range(24) if x not in (1, 6, 14, 10)]
    want = _codes(1, 0, [x for x in unknown if x < 10]) + _codes(1, 2, [x for x in unknown if x > 10])
    assert oracle.legal_actions(s, policy=1).tolist() == want
    assert oracle.legal_actions(s, policy=0).tolist() == _codes(1, 0, unknown) + _codes(1, 2, unknown)


def test_kept_guesses_with_jokers():
    # 26 tiles; opponent 1's row: 2, joker 24 (face down), 9 (face up), 15, joker 25 (face up), 20 (face up)
    # The joker slot (between face-up nothing on the left and 9 on the right) keeps numbered
    # identities below 9 and every unknown joker; slot 0 (tile 2) the same; slot 3 (tile 15)
    # lies between 9 and 20 (the face-up joker is not a numbered neighbour).
    row = [2, 24, 9, 15, 25, 20]
    s = encode([[4, 11, 22], row], {9, 25, 20}, cur=0, drawn=22, ntiles=26)
    unknown = [x for x in range(26) if x not in (4, 11, 22, 9, 25, 20)]
    below9 = [x for x in unknown if x < 9 or x >= 24]
    between = [x for x in unknown if 9 < x < 20 or x >= 24]
    want = _codes(1, 0, below9) + _codes(1, 1, below9) + _codes(1, 3, between)
    assert oracle.legal_actions(s, policy=1).tolist() == want


def test_own_tile_always_kept():
    cfgs = [oracle.OracleConfig(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5),
            oracle.OracleConfig(nplayers=4, ntiles=26, deal=3, max_predraw=8, max_revealed=3)]
    for cfg in cfgs:
        for st in oracle.init_states(cfg, 5, 200):
            d = decode(st)
            kept = set(oracle.legal_actions(st, policy=1).tolist())
            assert kept <= set(oracle.legal_actions(st, policy=0).tolist())
            for off in range(1, d["P"]):
                q = (d["cur"] + off) % d["P"]
                if not d["alive"][q]:
                    continue
                for i, t in enumerate(d["hands"][q]):
                    if t not in d["revealed"]:
                        assert (q << 10) | (i << 5) | t in kept


@pytest.mark.parametrize("name", sorted(ENDGAMES))
@pytest.mark.parametrize("cont", [0, 1 << 31])
def test_tiny_endgames_exact_ordered(name, cont):
    e = ENDGAMES[name]
    held = {t for h in e["hands"] for t in h}
    revealed = held - e["hidden"]
    exact = exact_win_probs(e["hands"], revealed, e["cur"], e["drawn"], e["T"], cont / 2 ** 32, ordered=True)
    assert sum(exact.values()) == 1
    plain = exact_win_probs(e["hands"], revealed, e["cur"], e["drawn"], e["T"], cont / 2 ** 32)
    assert exact != plain   # the policy changes the game's outcome distribution
    s = encode(e["hands"], revealed, cur=e["cur"], drawn=e["drawn"], ntiles=e["T"])
    cfg = oracle.OracleConfig(nplayers=len(e["hands"]), ntiles=e["T"], cont_thr=cont, policy=1)
    _mc_close(cfg, s, exact)
