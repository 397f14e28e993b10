"""Pins for the oracle's backpropagation (Sec. II-B, fourth step): which seat a
node's wins count, at every depth, in rollout mode and in value mode.

The positions are endgames solved by hand.  The pool is empty and every
player's face-down tiles are boxed in by face-up neighbours, so the searching
seat's view has exactly one consistent deal and every line of play has a
winner fixed in advance, whatever the random choices.  The game tree of each
position is written out below as data (actions in canonical order, the state
each one leads to, the winner of each finished line); the search over it is
textbook UCT (Sec. II-B; UCB1 with visits counted in playouts): expand the
first action without a child, else take the highest w/n + c sqrt(ln N) / sqrt(n)
(ties to the earliest action), stop expanding at depth d_max, credit each node
on the path with the leaf's wins of the seat that moved into it (the root: the
seat searching).  The oracle's whole node table must equal that model's.

A search that credited the searching seat at every node, or the seat to move
after a node's action, or the winner everywhere, fails these tables: the
depth-1 nodes of the 2-player endgame credit the loser of their line, the
depth-2 nodes credit the seat that is neither the searching seat nor the next
to move.
"""
import math

import numpy as np
import pytest

import oracle
from statefmt import encode


def g(q, slot, x):
    """Action code of a guess: seat << 10 | slot << 5 | identity."""
    return (q << 10) | (slot << 5) | x


# A position: ("pos", seat to move, winner of every playout from here,
#              [(action, next position), ...] in canonical order)
# A finished game: ("end", winner)
def pos(cur, playout_winner, moves):
    return ("pos", cur, playout_winner, moves)


def end(w):
    return ("end", w)


# ---- two players, 24 tiles ------------------------------------------------
# Seat 1 holds 0..11 with 4 and 5 face down (slots 4, 5, between face-up 3
# and 6); seat 0 holds 12..23 with 16 and 17 face down (slots 4, 5).  Seat 0
# to move.  A wrong guess turns the guesser's leftmost face-down tile up (the
# pool was empty at the draw); inside the tree a correct guess ends the turn.
# Seat 0 guessing right (4 in slot 4 or 5 in slot 5) wins in every line: seat
# 1 then either guesses wrong and is out, or guesses right and leaves seat 0 a
# single unknown tile.  Seat 0 guessing wrong loses: it has one face-down tile
# left and seat 1 knows it.


def _two_player_tree():
    after_p1_right_left = pos(0, 0, [(g(1, 5, 5), end(0))])   # seat 0 to find tile 5 in slot 5
    after_p1_right_right = pos(0, 0, [(g(1, 4, 4), end(0))])  # seat 0 to find tile 4 in slot 4
    a1 = pos(1, 0, [(g(0, 4, 16), after_p1_right_left), (g(0, 4, 17), end(0)),
                    (g(0, 5, 16), end(0)), (g(0, 5, 17), after_p1_right_left)])
    a4 = pos(1, 0, [(g(0, 4, 16), after_p1_right_right), (g(0, 4, 17), end(0)),
                    (g(0, 5, 16), end(0)), (g(0, 5, 17), after_p1_right_right)])
    a_wrong = pos(1, 1, [(g(0, 5, 17), end(1))])              # seat 0 has only 17 left, face down
    return pos(0, None, [(g(1, 4, 4), a1), (g(1, 4, 5), a_wrong), (g(1, 5, 4), a_wrong), (g(1, 5, 5), a4)])


def _two_player_root():
    h1 = list(range(0, 12))
    h0 = list(range(12, 24))
    revealed = (set(h0) - {16, 17}) | (set(h1) - {4, 5})
    return encode([h0, h1], revealed, cur=0, drawn=None, ntiles=24)


# ---- three players, 24 tiles ----------------------------------------------
# Seat 0 holds 16..23 (20 face down, slot 4), seat 1 holds 0..7 (4 face down,
# slot 4), seat 2 holds 8..15 (12 face down, slot 4); everything else is face
# up and the pool is empty.  Seat 0 to move; its unknown tiles are 4 and 12,
# and only 4 fits seat 1's slot, only 12 seat 2's.  Guessing seat 1's tile
# knocks seat 1 out and seat 2 then takes seat 0's last tile; guessing seat
# 2's tile knocks seat 2 out and seat 1 takes it; a wrong guess knocks seat 0
# itself out and seat 1 takes seat 2's tile.  Seat 0 loses every line.


def _three_player_tree():
    c1 = pos(2, 2, [(g(0, 4, 20), end(2))])
    c_wrong = pos(1, 1, [(g(2, 4, 12), end(1))])
    c4 = pos(1, 1, [(g(0, 4, 20), end(1))])
    return pos(0, None, [(g(1, 4, 4), c1), (g(1, 4, 12), c_wrong), (g(2, 4, 4), c_wrong), (g(2, 4, 12), c4)])


def _three_player_root():
    h0, h1, h2 = list(range(16, 24)), list(range(0, 8)), list(range(8, 16))
    revealed = set(range(24)) - {4, 12, 20}
    return encode([h0, h1, h2], revealed, cur=0, drawn=None, ntiles=24)


def _model(tree, observer, budget, playouts, d_max, credit, c=math.sqrt(2.0)):
    """Textbook UCT over an explicit game tree.  credit(position) gives the
    wins per seat of a fresh, unfinished leaf.  Returns node rows [action,
    parent, visits, wins] in creation order."""
    nodes = [dict(action=0, parent=-1, visits=0, wins=0, mover=observer, kids={}, pos=tree)]
    for _ in range(budget):
        k, depth = 0, 0
        path = [0]
        state = tree
        while state[0] == "pos" and depth < d_max:
            here = nodes[k]
            moves = state[3]
            fresh = next(((a, nxt) for a, nxt in moves if a not in here["kids"]), None)
            if fresh is not None:
                a, nxt = fresh
                nodes.append(dict(action=a, parent=k, visits=0, wins=0, mover=state[1], kids={}, pos=nxt))
                here["kids"][a] = len(nodes) - 1
                path.append(len(nodes) - 1)
                state = nxt
                break
            c_sqrt_ln = c * math.sqrt(math.log(here["visits"]))
            scored = []
            for a, nxt in moves:
                ch = nodes[here["kids"][a]]
                scored.append((ch["wins"] / ch["visits"] + c_sqrt_ln * (1.0 / math.sqrt(ch["visits"])),
                               (ch["wins"], ch["visits"]), a))
            best = scored[0]
            for sc in scored[1:]:
                # the model's log is libm's, the oracle's its own (2 ulp): a
                # near tie between different counts would make the pin fragile
                assert sc[1] == best[1] or abs(sc[0] - best[0]) > 1e-9, "near tie: choose another budget"
                if sc[0] > best[0]:
                    best = sc
            k = here["kids"][best[2]]
            path.append(k)
            state = nodes[k]["pos"]
            depth += 1
        wins = [0, 0, 0, 0]
        if state[0] == "end":
            wins[state[1]] = playouts
        else:
            wins = credit(state)
        for i in path:
            nodes[i]["visits"] += playouts
            nodes[i]["wins"] += wins[nodes[i]["mover"]]
    return np.array([[n["action"], n["parent"], n["visits"], n["wins"]] for n in nodes], dtype=np.int64)


CASES = {
    "2p": (_two_player_tree, _two_player_root, 2),
    "3p": (_three_player_tree, _three_player_root, 3),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("playouts,d_max,budget", [(1, 8, 40), (3, 8, 57), (2, 1, 30)])
def test_rollout_credit_by_mover_matches_hand_solved_tree(name, playouts, d_max, budget):
    tree_fn, root_fn, P = CASES[name]
    root = root_fn()
    assert oracle.det_count(root, 0) == 1                    # one consistent deal: the true one
    assert oracle.legal_actions(root).tolist() == [a for a, _ in tree_fn()[3]]
    cfg = oracle.OracleConfig(nplayers=P, ntiles=24, playouts=playouts, d_max=d_max, cont_thr=0)

    def playout_credit(state):
        w = [0, 0, 0, 0]
        w[state[2]] = playouts
        return w

    want = _model(tree_fn(), 0, budget, playouts, d_max, playout_credit)
    got, best = oracle.mcts(cfg, root, seed=5, tree=3, budget=budget)
    assert got.tolist() == want.tolist()
    # the decision: most visits among the root's children, ties to the first
    kids = want[want[:, 1] == 0]
    top = kids[np.argmax(kids[:, 2])]
    assert best.tolist() == [top[0], top[2], top[3], budget * playouts]


def test_hand_solved_trees_reach_depth_three_and_credit_every_seat():
    # the 2-player table has nodes at depths 1, 2 and 3 whose movers win and
    # lose; the 3-player table has depth-2 nodes moved into by seats 1 and 2
    cfg = oracle.OracleConfig(nplayers=2, ntiles=24, playouts=1, d_max=8, cont_thr=0)
    nodes, _ = oracle.mcts(cfg, _two_player_root(), seed=5, tree=3, budget=40)
    depth = [0] * len(nodes)
    for i in range(1, len(nodes)):
        depth[i] = depth[nodes[i][1]] + 1
    assert max(depth) == 3
    d1 = [i for i in range(len(nodes)) if depth[i] == 1]
    assert {nodes[i][3] == nodes[i][2] for i in d1} == {True, False}   # right guesses win, wrong lose
    d2 = [i for i in range(len(nodes)) if depth[i] == 2]
    assert {nodes[i][3] == 0 for i in d2} == {True, False}             # seat 1 loses under a right guess
    assert all(nodes[i][3] == nodes[i][2] for i in range(len(nodes)) if depth[i] == 3)
    cfg3 = oracle.OracleConfig(nplayers=3, ntiles=24, playouts=1, d_max=8)
    nodes3, _ = oracle.mcts(cfg3, _three_player_root(), seed=5, tree=3, budget=40)
    assert nodes3[0][3] == 0                                           # the searching seat never wins
    d2 = [i for i in range(1, len(nodes3)) if nodes3[nodes3[i][1]][1] == 0]
    assert d2 and all(nodes3[i][3] == nodes3[i][2] for i in d2)        # each credits its own mover


def _zero_hidden_params(b4):
    prm = np.zeros(oracle.value_nparams(), dtype=np.float32)
    prm[-4:] = b4
    return prm


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("playouts,d_max,budget", [(8, 8, 40), (16, 2, 33)])
def test_value_mode_credit_matches_hand_solved_tree(name, playouts, d_max, budget):
    # With every weight matrix zero the network's logits are its output bias,
    # so p over the seats in play, relative to the seat to move, is a softmax
    # of that bias in closed form; a fresh leaf credits absolute seat
    # (cur + r) mod P with round(p_r * playouts), a finished line its winner.
    tree_fn, root_fn, P = CASES[name]
    b4 = np.array([0.3, -0.5, 0.1, 2.0], dtype=np.float32)
    e = np.exp(b4[:P].astype(np.float64))
    p_rel = e / e.sum()
    frac = p_rel * playouts - np.floor(p_rel * playouts)
    assert (np.abs(frac - 0.5) > 0.01).all()                 # far from a rounding tie
    rel_credit = np.floor(p_rel * playouts + 0.5).astype(int)

    def value_credit(state):
        w = [0, 0, 0, 0]
        for r in range(P):
            w[(state[1] + r) % P] = int(rel_credit[r])
        return w

    cfg = oracle.OracleConfig(nplayers=P, ntiles=24, playouts=playouts, d_max=d_max, cont_thr=0)
    want = _model(tree_fn(), 0, budget, playouts, d_max, value_credit)
    got, _ = oracle.mcts(cfg, root_fn(), seed=5, tree=3, budget=budget, value_params=_zero_hidden_params(b4))
    assert got.tolist() == want.tolist()
    # value mode really changed the tables: the playout credit gives others
    want_roll = _model(tree_fn(), 0, budget, playouts, d_max,
                       lambda s: [playouts if q == s[2] else 0 for q in range(4)])
    assert want_roll.tolist() != want.tolist()
