"""GPU parity of vanilla MCTS-dvc (Sec. III-A): root children are
plausible-number sets, found through each tree's open-addressing table.
Trees, set counts and the summed decision against the oracle, bit for bit."""
import threading

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

VARIANTS = {
    "2p24": dict(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5),
    "3p24": dict(nplayers=3, ntiles=24, deal=4, max_predraw=6, max_revealed=3),
    "4p26j": dict(nplayers=4, ntiles=26, deal=3, max_predraw=8, max_revealed=3),
}


@pytest.fixture(scope="module")
def dvc():
    import paper_2403_10720_gb300 as m
    from paper_2403_10720_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return m


def _oracle(ocfg, roots, seed, budgets):
    out = {}

    def run(t):
        out[t] = oracle.mcts(ocfg, roots[t], seed, t, int(budgets[t]))

    ths = [threading.Thread(target=run, args=(t,)) for t in range(len(budgets))]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    return out


def _check(forest, stats, want):
    for t, (nodes, best) in want.items():
        exp = forest.dvc_tree_export(t).cpu().numpy()
        assert (exp[: len(nodes)] == nodes).all(), t
        assert (exp[len(nodes):] == -1).all(), t
        sets = int(((nodes[:, 1] == 0) & (nodes[:, 0] == oracle.SET)).sum())
        assert list(stats[t][:4]) == list(best), t
        assert stats[t][4] == sets and stats[t][5] == len(nodes), t


def _run(dvc, kw, budgets, seed, shape, root_seed=35):
    ocfg = oracle.OracleConfig(**kw)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    roots = ctx.dvc_init_states(root_seed, len(budgets))
    oroots = oracle.init_states(ocfg, root_seed, len(budgets))
    forest = dvc.Forest(ctx, roots, budgets, seed)
    forest.dvc_forest_tune(*shape)
    forest.dvc_mcts_step(max(budgets))
    stats = forest.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    return forest, stats, _oracle(ocfg, oroots, seed, budgets)


@pytest.mark.parametrize("variant,shape", [("2p24", (1, 0, 0, 0)), ("2p24", (2, 2, 8, 2)), ("3p24", (2, 3, 4, 1)),
                                           ("4p26j", (1, 0, 0, 0)), ("4p26j", (2, 2, 4, 2))])
def test_mcts_vanilla_bit_exact(dvc, variant, shape):
    kw = dict(VARIANTS[variant], playouts=16, vanilla=1)
    forest, stats, want = _run(dvc, kw, [150, 40, 1, 0, 97], 8, shape)
    _check(forest, stats, want)
    assert any(stats[t][4] > 1 for t in range(5))


@pytest.mark.parametrize("extra", [dict(d_max=0), dict(d_max=1), dict(tree_continue=1), dict(policy=1)])
def test_mcts_vanilla_options_bit_exact(dvc, extra):
    kw = dict(VARIANTS["2p24"], playouts=8, vanilla=1, **extra)
    forest, stats, want = _run(dvc, kw, [120, 64, 9], 3, (2, 2, 4, 2))
    _check(forest, stats, want)


def test_mcts_vanilla_split_steps_equal_fused(dvc):
    kw = dict(VARIANTS["4p26j"], playouts=16, vanilla=1)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    n, budget, P = 5, 50, 16
    roots = ctx.dvc_init_states(12, n)
    budgets = [budget, 30, 1, budget, 0]
    fused = dvc.Forest(ctx, roots, budgets, 3)
    fused.dvc_mcts_step(budget)
    split = dvc.Forest(ctx, roots, budgets, 3)
    leaves, tids, lids = split.dvc_forest_leaves()
    wins = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    for _ in range(budget + 2):
        split.dvc_mcts_select()
        split.dvc_mcts_expand()
        rc = dvc.lib().dvc_rollout_batch(ctx.h, leaves, n, P, 3, tids, lids, wins.data_ptr(), None, dvc._stream())
        assert rc == 0
        split.dvc_mcts_backprop(wins)
    ctx.dvc_check()
    for t in range(n):
        assert torch.equal(fused.dvc_tree_export(t), split.dvc_tree_export(t)), t
    assert torch.equal(fused.dvc_root_stats(), split.dvc_root_stats())


def test_mcts_vanilla_more_sets_than_12_bits(dvc):
    # an early four-player view has millions of plausible sets: with one
    # playout per iteration nearly every iteration opens a new one, past the
    # 4,095 children a 12-bit count could hold
    kw = dict(VARIANTS["4p26j"], max_predraw=0, playouts=1, vanilla=1, d_max=2)
    forest, stats, want = _run(dvc, kw, [4600, 4600], 5, (2, 2, 4, 1), root_seed=3)
    _check(forest, stats, want)
    assert stats[0][4] > 4095 and stats[1][4] > 4095


def test_server_rejects_vanilla(dvc):
    ctx = dvc.Context(dvc.Config(**dict(VARIANTS["2p24"], vanilla=1)), 0)
    with pytest.raises(Exception):
        dvc.Server(ctx, 1 << 28, 256, 0, 1)


def test_vanilla_against_mcts_dvc_games(dvc):
    from paper_2403_10720_gb300 import selfplay
    kw = dict(VARIANTS["2p24"], max_predraw=0, playouts=8)
    game = dvc.Context(dvc.Config(**kw), 0)
    van = dvc.Context(dvc.Config(**dict(kw, vanilla=1)), 0)
    a = selfplay.play_forest_agents(game, (van, 24), (game, 24), 12, root_seed=5, seed=3)
    b = selfplay.play_forest_agents(game, (van, 24), (game, 24), 12, root_seed=5, seed=3)
    assert a["games_finished"] == 12
    assert (a["winners"] == b["winners"]).all()   # every search is keyed: replays are identical
    assert a["decisions_a"] > 0 and a["decisions_b"] > 0


def test_vanilla_batched_sampled(dvc):
    """The benchmark's 4,096 batched two-player roots searched as vanilla
    trees (the bench's vanilla line: 256 iterations x 256 playouts), in the
    default pipeline shape; three trees replayed by the oracle, every tree
    checked for its counts."""
    from paper_2403_10720_gb300.workloads import BATCHED
    w = BATCHED
    kw = dict(w.config_kwargs(), vanilla=1)
    budget = 256
    ocfg = oracle.OracleConfig(**kw)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    roots = ctx.dvc_init_states(w.root_seed, w.n_trees)
    forest = dvc.Forest(ctx, roots, [budget] * w.n_trees, w.seed)
    forest.dvc_mcts_step(budget)
    stats = forest.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    assert (stats[:, 3] == budget * w.playouts).all() and (stats[:, 6] == budget).all()
    assert (stats[:, 4] >= 1).all() and (stats[:, 4] <= budget).all() and (stats[:, 7] == 0).all()
    oroots = oracle.init_states(ocfg, w.root_seed, w.n_trees)
    sample = [0, 1234, w.n_trees - 1]
    want = {}
    for t in sample:
        want[t] = oracle.mcts(ocfg, oroots[t], w.seed, t, budget)
    _check(forest, stats, want)
