"""Pins for vanilla MCTS-dvc (Sec. III-A): the root's children are
plausible-number sets -- one per distinct assignment of the tiles the observer
cannot see -- and the search below each is the usual guess tree."""
import numpy as np

import oracle
from statefmt import encode


def _key(det, obs):
    hands = [int.from_bytes(bytes(det[4 * p:4 * p + 4]), "little") for p in range(det[26]) if p != obs]
    hands += [0] * (3 - len(hands))
    return (hands[0] | hands[1] << 32, hands[2] | int(det[20]) << 32 | int(det[21]) << 40 | (int(det[22]) & 1) << 48)


def _check(cfg, root, seed, tree, budget):
    nodes, best = oracle.mcts(cfg, root, seed, tree, budget)
    obs = int(root[23])
    keys = [_key(oracle.determinize(cfg, root, obs, seed, tree, it), obs) for it in range(budget)]
    first = list(dict.fromkeys(keys))                      # distinct sets in first-sampled order
    sets = [i for i in range(len(nodes)) if nodes[i][1] == 0]
    assert all(nodes[i][0] == oracle.SET for i in sets)
    assert len(sets) == len(first)
    for i, k in zip(sets, first):                          # creation order and visits per set
        assert nodes[i][2] == cfg.playouts * keys.count(k)
    assert nodes[0][2] == cfg.playouts * budget
    # a set is entered on the observer's behalf: its wins are the observer's,
    # like the root's, and the sets partition the root's iterations
    assert sum(int(nodes[i][3]) for i in sets) == nodes[0][3]
    # the decision: visits summed per action over every set, ties to the lowest canonical rank
    tot = {}
    for a, par, v, w in nodes:
        if par >= 0 and nodes[par][1] == 0 and nodes[par][0] == oracle.SET:
            tot.setdefault(a, [0, 0])
            tot[a][0] += v
            tot[a][1] += w
    if tot:
        P = int(root[26])
        rank = lambda a: 0 if a == oracle.STOP else 1 + ((((a >> 10) - obs - 1) % P) << 10 | (a & 1023))  # noqa: E731
        want = min(tot, key=lambda a: (-tot[a][0], rank(a)))
        assert best[0] == want and best[1] == tot[want][0] and best[2] == tot[want][1]
    return nodes, sets


def test_sets_mid_game():
    cfg = oracle.OracleConfig(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5, playouts=8, vanilla=1)
    for t, root in enumerate(oracle.init_states(cfg, 12, 4)):
        nodes, sets = _check(cfg, root, 3, t, 300)
        assert len(sets) > 1


def test_sets_with_jokers():
    cfg = oracle.OracleConfig(nplayers=3, ntiles=26, deal=4, max_predraw=6, max_revealed=3, playouts=4, vanilla=1)
    for t, root in enumerate(oracle.init_states(cfg, 5, 3)):
        _check(cfg, root, 7, t, 200)


def test_single_deal_view_has_one_set():
    # every tile dealt, the observer's unknowns fill the opponent's face-down slots in order: one deal
    h0 = list(range(0, 24, 2))
    h1 = list(range(1, 24, 2))
    s = encode([h0, h1], {0, 2, 1, 7, 9}, cur=0, drawn=None, ntiles=24)
    assert oracle.det_count(s) == 1
    cfg = oracle.OracleConfig(nplayers=2, ntiles=24, deal=4, playouts=4, vanilla=1)
    nodes, sets = _check(cfg, s, 1, 0, 120)
    assert len(sets) == 1
    assert len(nodes) > 20   # the search goes on below the single set


def test_each_iteration_adds_one_node_and_a_new_set_is_a_leaf():
    # reading (c): an iteration whose determinization opens a new set adds
    # exactly that set node (its leaf is the determinized root); one that
    # finds its set adds at most one guess node below it
    cfg = oracle.OracleConfig(nplayers=2, ntiles=24, deal=4, max_predraw=6, max_revealed=5, playouts=4, vanilla=1)
    root = oracle.init_states(cfg, 21, 1)[0]
    obs = int(root[23])
    seen = set()
    prev = 1
    for b in range(1, 60):
        nodes, _ = oracle.mcts(cfg, root, 9, 0, b)
        key = _key(oracle.determinize(cfg, root, obs, 9, 0, b - 1), obs)
        added = len(nodes) - prev
        if key not in seen:
            assert added == 1 and nodes[-1][0] == oracle.SET and nodes[-1][1] == 0, b
            seen.add(key)
        else:
            assert added in (0, 1), b
            if added:
                assert nodes[-1][0] != oracle.SET and nodes[-1][1] != 0, b
        prev = len(nodes)
    nodes, _ = oracle.mcts(cfg, root, 9, 0, 1)
    assert nodes.shape[0] == 2 and nodes[1][0] == oracle.SET and nodes[0][2] == nodes[1][2] == 4


def test_joker_place_separates_sets():
    # the observer holds every tile but two; the opponent's two face-down
    # slots between its face-up 5 and 13 hold 9 and the black joker in an
    # order the observer cannot know: two consistent deals with the same
    # hands that differ only in where the joker stands -- two sets
    opp = [5, 24, 9, 13]
    own = [t for t in range(24) if t not in opp] + [25]
    s = encode([sorted(own[:-1]) + [25], opp], {5, 13}, cur=0, drawn=None, ntiles=26)
    assert oracle.det_count(s) == 2
    cfg = oracle.OracleConfig(nplayers=2, ntiles=26, deal=4, playouts=4, vanilla=1)
    nodes, sets = _check(cfg, s, 3, 0, 60)
    assert len(sets) == 2
