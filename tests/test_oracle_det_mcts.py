"""Pins for the oracle's determinizer (Sec. III-A, plausible numbers) and its
UCT search (Sec. II-B four steps; Sec. III-A simplifications; UCB1)."""
import math
from collections import Counter

import numpy as np
import pytest

import oracle
from bruteforce import consistent_deals
from statefmt import decode, encode


def _mk_view(T, observer, opps, pool):
    """opps: {seat: (left-to-right tiles, face-down subset)}; the observer
    holds every other tile, face down."""
    P = len(opps) + 1
    used = set(pool)
    for seq, _ in opps.values():
        used |= set(seq)
    own = sorted(t for t in range(T) if t not in used)
    hands = [None] * P
    hidden = set(own)
    for q, (seq, hid) in opps.items():
        hands[q] = list(seq)
        hidden |= set(hid)
    hands[observer] = own
    return dict(hands=hands, hidden=hidden, cur=observer, T=T)


VIEWS = {
    # 2 players, 24 tiles: opponent 1 has anchors 6 and 15 face up
    "2p": _mk_view(24, 0, {1: ([2, 6, 9, 13, 15, 22], {2, 9, 13, 22})}, {1, 4, 10, 12, 17}),
    # 3 players, 26 tiles, the white joker face down in player 2's hand
    "3p_joker": _mk_view(26, 0, {1: ([3, 12, 14, 18], {3, 14, 18}), 2: ([5, 25, 16, 21], {5, 25, 21})},
                         {24, 7}),
    # 4 players, 26 tiles, both jokers unknown to the observer (one in the pool)
    "4p_jokers": _mk_view(26, 0, {1: ([0, 24, 11], {0, 24}), 2: ([6, 13], {13}), 3: ([7, 19, 23], {7, 19})},
                          {25, 2}),
}


def _view(name):
    v = VIEWS[name]
    held = {t for h in v["hands"] for t in h}
    revealed = held - v["hidden"]
    s = encode(v["hands"], revealed, cur=v["cur"], drawn=None, ntiles=v["T"])
    return v, revealed, s


@pytest.mark.parametrize("name", sorted(VIEWS))
def test_det_count_matches_enumeration(name):
    v, revealed, s = _view(name)
    deals = consistent_deals(v["hands"], revealed, v["cur"], v["T"])
    assert len(deals) > 3
    assert oracle.det_count(s, v["cur"]) == len(deals)


@pytest.mark.parametrize("name", sorted(VIEWS))
def test_determinize_uniform_and_consistent(name):
    from scipy.stats import chisquare
    v, revealed, s = _view(name)
    deals = consistent_deals(v["hands"], revealed, v["cur"], v["T"])
    index = {d: i for i, d in enumerate(deals)}
    P = len(v["hands"])
    opps = [(v["cur"] + k) % P for k in range(1, P)]
    cfg = oracle.OracleConfig(nplayers=P, ntiles=v["T"])
    n = max(20 * len(deals), 4000)
    counts = Counter()
    for it in range(n):
        out = decode(oracle.determinize(cfg, s, v["cur"], seed=123, tree=4, it=it))
        assert out["hands"][v["cur"]] == v["hands"][v["cur"]]
        assert out["revealed"] == revealed
        for q in range(P):
            assert len(out["hands"][q]) == len(v["hands"][q])
            for i, t in enumerate(v["hands"][q]):
                if t in revealed:
                    assert out["hands"][q][i] == t
        key = tuple(tuple(t for i, t in enumerate(out["hands"][q]) if v["hands"][q][i] not in revealed)
                    for q in opps)
        assert key in index
        counts[index[key]] += 1
    obs = np.array([counts[i] for i in range(len(deals))])
    assert chisquare(obs).pvalue > 1e-4


def test_determinize_deterministic_per_iteration():
    v, revealed, s = _view("3p_joker")
    cfg = oracle.OracleConfig(nplayers=3, ntiles=26)
    a = oracle.determinize(cfg, s, 0, seed=9, tree=2, it=17)
    b = oracle.determinize(cfg, s, 0, seed=9, tree=2, it=17)
    assert (a == b).all()


def _toy_root():
    # Player 1 hides only tile 5, boxed in by face-up 4 and 6, so every
    # determinization is the true deal.  Player 0's only face-down tile is the
    # one it just drew (23); tile 20 is in the pool.  Player 0 has two guesses:
    # (slot 5, tile 5) wins at once, (slot 5, tile 20) loses at once.
    h1 = list(range(0, 12))
    h0 = [12, 13, 14, 15, 16, 17, 18, 19, 21, 22, 23]
    revealed = (set(h0) - {23}) | (set(h1) - {5})
    return encode([h0, h1], revealed, cur=0, drawn=23, ntiles=24)


def test_uct_forced_win_sequence():
    # Textbook UCB1 (visits in playouts, one playout per iteration): the first
    # two iterations expand both actions in canonical order, then each picks
    # argmax w/n + sqrt(2) sqrt(ln N / n).
    root = _toy_root()
    assert oracle.legal_count(root) == 2
    budget = 200
    cfg = oracle.OracleConfig(playouts=1)
    nodes, best = oracle.mcts(cfg, root, seed=1, tree=0, budget=budget)
    win, lose = (1 << 10) | (5 << 5) | 5, (1 << 10) | (5 << 5) | 20
    nA, wA, nB = 1, 1, 1
    seq = []
    for it in range(2, budget):
        N = it
        sA = wA / nA + math.sqrt(2) * math.sqrt(math.log(N) / nA)
        sB = 0.0 + math.sqrt(2) * math.sqrt(math.log(N) / nB)
        assert abs(sA - sB) > 1e-9
        if sA > sB:
            nA += 1
            wA += 1
            seq.append("A")
        else:
            nB += 1
            seq.append("B")
    assert "B" in seq[2:]
    assert nodes.shape == (3, 4)
    assert nodes[0].tolist() == [0, -1, budget, nodes[0][3]]
    assert nodes[1].tolist() == [win, 0, nA, wA]
    assert nodes[2].tolist() == [lose, 0, nB, 0]
    assert best.tolist() == [win, nA, wA, budget]


CFG1 = oracle.OracleConfig(nplayers=2, ntiles=24, deal=4, max_predraw=0, playouts=1)


@pytest.mark.parametrize("playouts,d_max", [(1, 8), (4, 2), (3, 1)])
def test_mcts_count_invariants(playouts, d_max):
    cfg = oracle.OracleConfig(nplayers=2, ntiles=24, deal=4, max_predraw=10, playouts=playouts, d_max=d_max)
    roots = oracle.init_states(cfg, seed=2, n=3)
    budget = 300
    for t, r in enumerate(roots):
        nodes, best = oracle.mcts(cfg, r, seed=7, tree=t, budget=budget)
        assert nodes[0][2] == playouts * budget                 # I8: root visits
        assert len(nodes) <= budget + 1
        child_sum = np.zeros(len(nodes), dtype=np.int64)
        depth = np.zeros(len(nodes), dtype=np.int64)
        for i in range(1, len(nodes)):
            a, par, vis, w = nodes[i]
            assert 0 <= par < i
            depth[i] = depth[par] + 1
            assert depth[i] <= d_max
            child_sum[par] += vis
            assert 0 <= w <= vis and vis % playouts == 0 and vis > 0
        assert child_sum[0] == nodes[0][2]
        stop = nodes[:, 2] - child_sum
        assert (stop[1:] >= playouts).all() and (stop % playouts == 0).all()
        kids = nodes[nodes[:, 1] == 0]
        bi = np.argmax(kids[:, 2])
        assert best[1] == kids[:, 2].max() and best[3] == playouts * budget
        # siblings carry distinct actions
        for par in set(nodes[1:, 1].tolist()):
            acts = nodes[nodes[:, 1] == par][:, 0]
            assert len(set(acts.tolist())) == len(acts)


def test_mcts_expands_canonically_then_selects():
    # With a fixed budget smaller than the root's legal count, every iteration
    # expands a new root child, in canonical order (opponent, slot, identity).
    r = oracle.init_states(CFG1, seed=1, n=1)[0]
    L = oracle.legal_count(r)
    nodes, _ = oracle.mcts(CFG1, r, seed=1, tree=0, budget=L)
    acts = nodes[1:, 0].tolist()
    assert all(p == 0 for p in nodes[1:, 1])
    assert acts == sorted(acts) and len(acts) == L


def test_mcts_decision_prefers_winning_guess():
    root = _toy_root()
    for P in (1, 8):
        cfg = oracle.OracleConfig(playouts=P)
        _, best = oracle.mcts(cfg, root, seed=3, tree=1, budget=64)
        assert best[0] == (1 << 10) | (5 << 5) | 5


def test_mcts_work_counts_one_step_per_guess():
    # With d_max = 0 every iteration's leaf is the determinized root, so the
    # search's game steps are the traced playouts' lengths (one record per
    # guess), plus one per playout for the continue coin a may-stop leaf
    # draws first.
    P, budget, seed, tree = 3, 5, 4, 2
    cfg = oracle.OracleConfig(playouts=P, d_max=0, max_predraw=6)
    root = oracle.init_states(cfg, 9, 1)[0]
    want = 0
    for it in range(budget):
        leaf = oracle.determinize(cfg, root, int(root[23]), seed, tree, it)
        want += sum(len(oracle.playout_trace(cfg, leaf, seed, tree, j, it)) for j in range(P))
    words, steps = oracle.mcts_work(cfg, root, seed, tree, budget)
    assert steps == want and words >= steps
    # a may-stop root: the coin first
    ms = root.copy()
    ms[22] |= 2
    cfg_c = oracle.OracleConfig(playouts=P, d_max=0, tree_continue=1)
    want = budget * P
    for it in range(budget):
        leaf = oracle.determinize(cfg_c, ms, int(ms[23]), seed, tree, it)
        assert leaf[22] & 2
        want += sum(len(oracle.playout_trace(cfg_c, leaf, seed, tree, j, it)) for j in range(P))
    assert oracle.mcts_work(cfg_c, ms, seed, tree, budget)[1] == want


@pytest.mark.parametrize("vanilla", [0, 1])
def test_root_merge_of_one_tree_is_its_decision(vanilla):
    # Sec. III-B: merging a single search reproduces its own decision
    cfg = oracle.OracleConfig(nplayers=2, ntiles=24, deal=4, max_predraw=10, playouts=3, vanilla=vanilla)
    for t, r in enumerate(oracle.init_states(cfg, seed=12, n=3)):
        nodes, best = oracle.mcts(cfg, r, seed=4, tree=t, budget=150)
        assert oracle.root_merge(r, [nodes], vanilla).tolist() == best.tolist()


def test_root_merge_sums_over_trees_hand_made():
    root = _toy_root()                                  # seat 0 to move, 2 players
    a1, a2 = (1 << 10) | (2 << 5) | 3, (1 << 10) | (0 << 5) | 5
    # rows [action, parent, visits, wins]; row 0 the root; a grandchild (parent 1) is not a root action
    A = [[0, -1, 10, 4], [a1, 0, 6, 1], [a2, 0, 4, 3], [a2, 1, 99, 0]]
    B = [[0, -1, 10, 2], [a2, 0, 7, 2], [a1, 0, 3, 0]]
    assert oracle.root_merge(root, [A]).tolist() == [a1, 6, 1, 10]
    assert oracle.root_merge(root, [B]).tolist() == [a2, 7, 2, 10]
    assert oracle.root_merge(root, [A, B]).tolist() == [a2, 11, 5, 20]     # 4 + 7 against 6 + 3
    # a tie in summed visits goes to the lower canonical rank: a2 (slot 0) before a1 (slot 2)
    C = [[0, -1, 10, 0], [a1, 0, 5, 5], [a2, 0, 5, 0]]
    assert oracle.root_merge(root, [C]).tolist() == [a2, 5, 0, 10]
    # vanilla tables: the set nodes (children of the root) are summed over
    V = [[0, -1, 12, 3], [0xFFE, 0, 8, 2], [a1, 1, 5, 2], [a2, 1, 3, 0], [0xFFE, 0, 4, 1], [a2, 4, 4, 1]]
    assert oracle.root_merge(root, [V], vanilla=1).tolist() == [a2, 7, 1, 12]
