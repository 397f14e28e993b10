"""Pins for the oracle's full game tree (Fig. 2a): after a correct guess the
player keeps the turn and may STOP or guess again."""
import numpy as np
import pytest

import oracle
from bruteforce import exact_win_probs
from statefmt import decode, encode
from test_oracle_play import GAME, HANDS, REV, SEED, TURN, _expected_draw
from test_oracle_rules import ENDGAMES, _mc_close

STOP = oracle.STOP


def _pos(may_stop=False):
    return encode(HANDS, REV, cur=0, drawn=6, ntiles=24, may_stop=may_stop)


def test_correct_guess_keeps_the_turn():
    rc, out = oracle.play_move(_pos(), (1 << 10) | (0 << 5) | 3, SEED, GAME, TURN, cont=1)
    d = decode(out)
    assert rc == 0 and d["cur"] == 0 and d["may_stop"] and d["drawn"] == 6
    assert d["revealed"] == REV | {3} and d["hands"][1] == [3, 10, 17]   # nobody drew
    # ... then STOP: the turn passes and the next seat draws from the play stream
    rc, out2 = oracle.play_move(out, STOP, SEED, GAME, TURN, cont=1)
    d2 = decode(out2)
    assert rc == 0 and d2["cur"] == 1 and not d2["may_stop"] and d2["drawn"] == _expected_draw(HANDS)
    # ... or a wrong guess after it: the tile drawn this turn turns face up
    rc, out3 = oracle.play_move(out, (1 << 10) | (2 << 5) | 18, SEED, GAME, TURN, cont=1)
    d3 = decode(out3)
    assert rc == 0 and d3["cur"] == 1 and not d3["may_stop"] and d3["revealed"] == REV | {3, 6}


def test_stop_only_when_allowed():
    rc, out = oracle.play_move(_pos(), STOP, SEED, GAME, TURN, cont=1)
    assert rc == -1 and (out == _pos()).all()
    # with cont = 0 a correct guess still ends the turn (Sec. III-A)
    rc, out = oracle.play_move(_pos(), (1 << 10) | (0 << 5) | 3, SEED, GAME, TURN, cont=0)
    assert decode(out)["cur"] == 1 and not decode(out)["may_stop"]


@pytest.mark.parametrize("name", sorted(ENDGAMES))
@pytest.mark.parametrize("cont", [0, 1 << 31])
def test_playout_from_may_stop_state(name, cont):
    """A playout that starts where the mover may stop first draws the continue coin."""
    e = ENDGAMES[name]
    held = {t for h in e["hands"] for t in h}
    revealed = held - e["hidden"]
    exact = exact_win_probs(e["hands"], revealed, e["cur"], e["drawn"], e["T"], cont / 2 ** 32, may_stop=True)
    assert sum(exact.values()) == 1
    s = encode(e["hands"], revealed, cur=e["cur"], drawn=e["drawn"], ntiles=e["T"], may_stop=True)
    cfg = oracle.OracleConfig(nplayers=len(e["hands"]), ntiles=e["T"], cont_thr=cont)
    _mc_close(cfg, s, exact)


def _tree(cont, budget=400, P=8):
    cfg = oracle.OracleConfig(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5, playouts=P,
                              tree_continue=cont)
    root = oracle.init_states(cfg, 9, 1)[0]
    return oracle.mcts(cfg, root, 4, 0, budget)


def test_full_tree_structure():
    nodes, best = _tree(1)
    action, parent = nodes[:, 0], nodes[:, 1]
    stops = np.nonzero(action == STOP)[0]
    assert len(stops) > 0                      # correct in-tree guesses lead to may-stop nodes
    for i in stops:
        p = parent[i]
        assert p > 0 and action[p] != STOP     # below a guess, never below the root or another STOP
    # (a guess node's children mix the actions of the guesser, who went on in
    # determinizations where the guess was right, and of the next seat, who
    # moves where it was wrong; with two players their guess codes differ)
    # visit counts: the root has P x budget; a child never exceeds its parent
    assert nodes[0][2] == 8 * 400
    for i in range(1, len(nodes)):
        assert nodes[i][2] <= nodes[parent[i]][2]
    plain, _ = _tree(0)
    assert not (plain[:, 0] == STOP).any()
    assert len(plain) != len(nodes) or (plain != nodes).any()
