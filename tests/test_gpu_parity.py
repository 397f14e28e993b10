"""GPU parity: every entry point of libdvc against the CPU oracle, bit for bit.

All inputs are seeded and synthetic.  Integer game logic and the UCT
decisions are compared exactly (the method has no tolerance to give: states,
win counts, visit counts and decisions are integers, and the UCT score is
computed with the same IEEE single-precision operations on both sides).
"""
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_2403_10720_gb300.workloads import BATCHED, SINGLE_TREE, UNEVEN

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


def _ctx(dvc, **kw):
    return dvc.Context(dvc.Config(**kw), 0)


def _u32(a):
    return torch.from_numpy(np.asarray(a, dtype=np.uint32).view(np.int32)).cuda()


def test_philox_matches_reference_and_oracle(dvc):
    ctx = _ctx(dvc)
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(4096, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    mine = ctx.dvc_philox(_u32(ctr), _u32(key), False).cpu().numpy().view(np.uint32)
    ref = ctx.dvc_philox(_u32(ctr), _u32(key), True).cpu().numpy().view(np.uint32)
    assert (mine == ref).all()
    for i in range(0, 4096, 97):
        assert list(mine[i]) == oracle.philox4x32_10(ctr[i], key[i])


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("n", [1, 333])
def test_init_states_bit_exact(dvc, variant, n):
    kw = VARIANTS[variant]
    ctx = _ctx(dvc, **kw)
    got = ctx.dvc_init_states(99, n).cpu().numpy()
    want = oracle.init_states(oracle.OracleConfig(**kw), 99, n)
    assert (got == want).all()


def test_init_states_empty(dvc):
    ctx = _ctx(dvc)
    out = torch.zeros((1, 32), dtype=torch.uint8, device="cuda")
    ctx.dvc_init_states(3, 0, out=out)
    assert int(out.sum()) == 0


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_determinize_bit_exact(dvc, variant):
    kw = VARIANTS[variant]
    ocfg = oracle.OracleConfig(**kw)
    roots = oracle.init_states(ocfg, 7, 300)
    n = len(roots)
    rng = np.random.default_rng(1)
    tree = rng.integers(0, 1 << 20, size=n).astype(np.uint32)
    it = rng.integers(0, 1 << 20, size=n).astype(np.uint32)
    ctx = _ctx(dvc, **kw)
    got = ctx.dvc_determinize(torch.from_numpy(roots).cuda(), -1, 31, _u32(tree), _u32(it)).cpu().numpy()
    ctx.dvc_check()
    for i in range(n):
        want = oracle.determinize(ocfg, roots[i], -1, 31, int(tree[i]), int(it[i]))
        assert (got[i] == want).all(), i


def test_determinize_joker_views(dvc):
    from test_oracle_det_mcts import VIEWS, _view
    for name in sorted(VIEWS):
        v, revealed, s = _view(name)
        P = len(v["hands"])
        ocfg = oracle.OracleConfig(nplayers=P, ntiles=v["T"])
        ctx = _ctx(dvc, nplayers=P, ntiles=v["T"], deal=2)
        n = 512
        roots = torch.from_numpy(np.tile(s, (n, 1))).cuda()
        its = np.arange(n, dtype=np.uint32)
        got = ctx.dvc_determinize(roots, v["cur"], 5, _u32(np.full(n, 3)), _u32(its)).cpu().numpy()
        for i in range(0, n, 7):
            want = oracle.determinize(ocfg, s, v["cur"], 5, 3, i)
            assert (got[i] == want).all(), (name, i)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("P", [1, 37, 64])
def test_rollout_bit_exact(dvc, variant, P):
    kw = VARIANTS[variant]
    ocfg = oracle.OracleConfig(**kw)
    leaves = oracle.init_states(ocfg, 13, 45)
    n = len(leaves)
    tree = np.arange(n, dtype=np.uint32) * 3 + 1
    leaf = np.arange(n, dtype=np.uint32) * 7 + 2
    ctx = _ctx(dvc, **kw)
    words = torch.zeros(1, dtype=torch.int64, device="cuda")
    wins = ctx.dvc_rollout_batch(torch.from_numpy(leaves).cuda(), P, 77, _u32(tree), _u32(leaf), words=words)
    wins = wins.cpu().numpy()
    total = 0
    for i in range(n):
        w, wd = oracle.rollout(ocfg, leaves[i], P, 77, int(tree[i]), int(leaf[i]))
        assert (wins[i] == w).all(), i
        total += wd
    assert int(words.item()) == total


def test_rollout_finished_leaves(dvc):
    kw = VARIANTS["2p24"]
    leaves = oracle.init_states(oracle.OracleConfig(**kw), 1, 3).copy()
    leaves[0, 28] = 1      # already won by seat 1
    leaves[2, 28] = 0xFE   # inactive marker: no credit
    ctx = _ctx(dvc, **kw)
    wins = ctx.dvc_rollout_batch(torch.from_numpy(leaves).cuda(), 10, 1, _u32([0, 1, 2]), _u32([0, 0, 0]))
    wins = wins.cpu().numpy()
    assert wins[0].tolist() == [0, 10, 0, 0]
    assert wins[1].sum() == 10
    assert wins[2].tolist() == [0, 0, 0, 0]


def _oracle_trees(ocfg, roots, seed, budgets, trees, tree_ids=None):
    out = {}

    def run(t):
        tid = t if tree_ids is None else int(tree_ids[t])
        out[t] = oracle.mcts(ocfg, roots[t], seed, tid, int(budgets[t]))

    ths = [threading.Thread(target=run, args=(t,)) for t in trees]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    return out


def _check_forest(forest, stats, want, trees):
    for t in trees:
        nodes, best = want[t]
        exp = forest.dvc_tree_export(t).cpu().numpy()
        assert (exp[: len(nodes)] == nodes).all(), t
        assert (exp[len(nodes):] == -1).all(), t
        assert stats[t][0] == best[0] and stats[t][1] == best[1] and stats[t][2] == best[2], t
        assert stats[t][3] == best[3] and stats[t][5] == len(nodes), t


@pytest.mark.parametrize("variant,P,budgets", [
    ("2p24", 32, [200, 57, 1, 0, 120, 200]),
    ("3p24", 16, [150, 90, 3]),
    ("4p26j", 32, [120, 64, 200, 17]),
    ("2p24", 256, [40, 33]),
])
def test_mcts_fused_bit_exact(dvc, variant, P, budgets):
    kw = dict(VARIANTS[variant], playouts=P)
    ocfg = oracle.OracleConfig(**kw)
    n = len(budgets)
    ctx = _ctx(dvc, **kw)
    roots = ctx.dvc_init_states(21, n)
    oroots = oracle.init_states(ocfg, 21, n)
    assert (roots.cpu().numpy() == oroots).all()
    tree_ids = np.arange(n, dtype=np.uint32) * 5 + 9
    forest = dvc.Forest(ctx, roots, budgets, 8, tree_ids=tree_ids)
    forest.dvc_mcts_step(max(budgets))
    stats = forest.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    assert (stats[:, 6] == np.asarray(budgets)).all()
    want = _oracle_trees(ocfg, oroots, 8, budgets, range(n), tree_ids)
    _check_forest(forest, stats, want, range(n))


def test_mcts_steps_compose(dvc):
    kw = dict(VARIANTS["2p24"], playouts=32)
    ctx = _ctx(dvc, **kw)
    roots = ctx.dvc_init_states(4, 5)
    a = dvc.Forest(ctx, roots, [150] * 5, 6)
    a.dvc_mcts_step(150)
    b = dvc.Forest(ctx, roots, [150] * 5, 6)
    for _ in range(3):
        b.dvc_mcts_step(50)
    b.dvc_mcts_step(50)   # budget spent: no-op
    for t in range(5):
        assert torch.equal(a.dvc_tree_export(t), b.dvc_tree_export(t))
    assert torch.equal(a.dvc_root_stats(), b.dvc_root_stats())


@pytest.mark.parametrize("variant,P", [("2p24", 64), ("4p26j", 32)])
def test_mcts_split_steps_equal_fused(dvc, variant, P):
    kw = dict(VARIANTS[variant], playouts=P)
    ctx = _ctx(dvc, **kw)
    n, budget = 7, 60
    roots = ctx.dvc_init_states(12, n)
    budgets = [budget, 30, budget, 1, budget, 45, 0]
    fused = dvc.Forest(ctx, roots, budgets, 3)
    fused.dvc_mcts_step(budget)
    split = dvc.Forest(ctx, roots, budgets, 3)
    leaves, tids, lids = split.dvc_forest_leaves()
    wins = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    for _ in range(budget + 2):
        split.dvc_mcts_select()
        split.dvc_mcts_expand()
        rc = dvc.lib().dvc_rollout_batch(ctx.h, leaves, n, P, 3, tids, lids, wins.data_ptr(), None,
                                         dvc._stream())
        assert rc == 0
        split.dvc_mcts_backprop(wins)
    ctx.dvc_check()
    for t in range(n):
        assert torch.equal(fused.dvc_tree_export(t), split.dvc_tree_export(t)), t
    assert torch.equal(fused.dvc_root_stats(), split.dvc_root_stats())


def test_single_tree_workload(dvc):
    w = SINGLE_TREE
    kw = w.config_kwargs()
    ocfg = oracle.OracleConfig(**kw)
    ctx = _ctx(dvc, **kw)
    roots = ctx.dvc_init_states(w.root_seed, 1)
    forest = dvc.Forest(ctx, roots, w.budgets(), w.seed)
    forest.dvc_mcts_step(w.budget)
    stats = forest.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    oroots = oracle.init_states(ocfg, w.root_seed, 1)
    want = _oracle_trees(ocfg, oroots, w.seed, w.budgets(), [0])
    _check_forest(forest, stats, want, [0])


def test_batched_workload_full_size_sampled(dvc):
    """The full 4,096-tree x 4,096-iteration x 256-playout batch as the
    benchmark launches it; three trees are replayed by the oracle and every
    tree is checked for the visit-count invariants."""
    w = BATCHED
    kw = w.config_kwargs()
    ocfg = oracle.OracleConfig(**kw)
    ctx = _ctx(dvc, **kw)
    roots = ctx.dvc_init_states(w.root_seed, w.n_trees)
    forest = dvc.Forest(ctx, roots, w.budgets(), w.seed)
    forest.dvc_mcts_step(w.budget)
    stats = forest.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    assert (stats[:, 3] == w.budget * w.playouts).all()
    assert (stats[:, 6] == w.budget).all()
    assert (stats[:, 5] <= w.budget + 1).all() and (stats[:, 7] == 0).all()
    sample = [0, 1234, w.n_trees - 1]
    oroots = oracle.init_states(ocfg, w.root_seed, w.n_trees)
    assert (roots.cpu().numpy() == oroots).all()
    want = _oracle_trees(ocfg, oroots, w.seed, w.budgets(), sample)
    _check_forest(forest, stats, want, sample)


def test_uneven_workload_sampled(dvc):
    """The 4-player joker forest at reduced size: 64 trees with the
    workload's log-uniform budgets capped at 3,000, four replayed."""
    w = UNEVEN
    kw = w.config_kwargs()
    ocfg = oracle.OracleConfig(**kw)
    ctx = _ctx(dvc, **kw)
    n = 64
    budgets = np.minimum(w.budgets(n), 3000)
    roots = ctx.dvc_init_states(w.root_seed, n)
    forest = dvc.Forest(ctx, roots, budgets, w.seed)
    forest.dvc_mcts_step(int(budgets.max()))
    stats = forest.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    assert (stats[:, 6] == budgets).all()
    oroots = oracle.init_states(ocfg, w.root_seed, n)
    sample = [0, 5, 17, 63]
    want = _oracle_trees(ocfg, oroots, w.seed, budgets, sample)
    _check_forest(forest, stats, want, sample)


def test_uneven_workload_full_budgets_sampled(dvc):
    """The whole uneven forest -- 16,384 four-player joker trees, budgets
    log-uniform in 1k-100k -- searched to the end of every budget under the
    library's schedule (the autotuned pipeline shape; from the iteration at
    which at most 16 trees per SM still run, fused CTAs of 4 trees repacked
    with running trees every 2,000 iterations; from at most 5 per SM, one tree
    per CTA), then trees replayed by the oracle at their real budgets: the
    largest (about 100k iterations, so the largest arenas and child blocks),
    two that end just before and just after the switch to the fused engine,
    and three more.  Node tables and decisions bit-exact."""
    from paper_2403_10720_gb300 import autotune
    w = UNEVEN
    kw = w.config_kwargs()
    ocfg = oracle.OracleConfig(**kw)
    ctx = _ctx(dvc, **kw)
    n = w.n_trees
    budgets = w.budgets(n)
    roots = ctx.dvc_init_states(w.root_seed, n)
    forest = dvc.Forest(ctx, roots, budgets, w.seed)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cut = autotune.tail_start(budgets, sms, autotune.PACK_TREES_PER_SM)   # pipeline -> packed fused CTAs
    assert cut is not None and 0 < cut < int(budgets.max())
    assert 0 < cut < autotune.tail_start(budgets, sms) < int(budgets.max())
    autotune.step_with_tail(forest, budgets, (2, 1, 1, 16), sms)
    stats = forest.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    assert (stats[:, 6] == budgets).all()
    order = np.argsort(budgets)
    sample = [int(order[-1])]                                           # the longest budget
    sample += [int(order[np.searchsorted(budgets[order], cut) - 1]),   # ends just before the switch
               int(order[np.searchsorted(budgets[order], cut, side="right")])]  # just after it
    rng = np.random.default_rng(9)
    sample += [int(t) for t in rng.choice(n, size=3, replace=False)]
    oroots = oracle.init_states(ocfg, w.root_seed, n)
    want = _oracle_trees(ocfg, oroots, w.seed, budgets, sample)
    _check_forest(forest, stats, want, sample)
    forest.close()


@pytest.mark.parametrize("variant,engine_shape", [("4p26j", (1, 4, 4, 0)), ("2p24", (1, 3, 2, 0)),
                                                  ("4p26j", (2, 2, 1, 3))])
def test_caller_order_and_active_prefix(dvc, variant, engine_shape):
    """dvc_forest_order: a forest searched in chunks, its running trees
    repacked before each chunk (running first, longest remaining budget
    first; the fused engine visits only those), gives the same trees and
    decisions as one step with the default order; trees sampled against the
    oracle.  A non-permutation or an out-of-range prefix is refused."""
    from paper_2403_10720_gb300 import autotune
    kw = dict(VARIANTS[variant], playouts=16)
    ctx = _ctx(dvc, **kw)
    n = 97
    rng = np.random.default_rng(17)
    budgets = rng.integers(1, 160, size=n).astype(np.int32)
    roots = ctx.dvc_init_states(23, n)
    a = dvc.Forest(ctx, roots, budgets, 19)
    a.dvc_mcts_step(int(budgets.max()))
    b = dvc.Forest(ctx, roots, budgets, 19)
    b.dvc_forest_tune(*engine_shape)
    autotune._packed_steps(b, budgets, 0, int(budgets.max()), chunk=37)
    sa, sb = a.dvc_root_stats().cpu().numpy(), b.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    assert (sa == sb).all() and (sb[:, 6] == budgets).all()
    for t in (0, 48, 96):
        assert torch.equal(a.dvc_tree_export(t), b.dvc_tree_export(t))
    ocfg = oracle.OracleConfig(**kw)
    oroots = oracle.init_states(ocfg, 23, n)
    want = _oracle_trees(ocfg, oroots, 19, budgets, [int(np.argmax(budgets)), 5])
    _check_forest(b, sb, want, [int(np.argmax(budgets)), 5])
    bad = np.arange(n, dtype=np.int32)
    bad[3] = 4
    for order, k in ((bad, 0), (np.arange(n, dtype=np.int32), n + 1), (np.arange(n, dtype=np.int32), -1)):
        with pytest.raises(dvc.DvcError):
            b.dvc_forest_order(order, k)
    b.dvc_forest_order(None)                                   # the default order again
    assert dvc.lib().dvc_forest_order(b.h, None, 5) == -1     # the default order runs every tree
    b.dvc_forest_reset()
    b.dvc_mcts_step(int(budgets.max()))
    assert (b.dvc_root_stats().cpu().numpy() == sa).all()
    ctx.dvc_check()
    a.close()
    b.close()


@pytest.mark.parametrize("variant,shape", [
    ("4p26j", (1, 3, 2, 0)), ("4p26j", (1, 5, 8, 0)), ("4p26j", (1, 2, 1, 0)), ("4p26j", (1, 7, 3, 0)),
    ("4p26j", (2, 3, 2, 1)), ("4p26j", (2, 5, 32, 2)), ("4p26j", (2, 1, 4, 4)), ("4p26j", (2, 2, 2, 3)),
    # two players, 24 tiles: the playout fast path with its shared-memory word rings
    ("2p24", (2, 3, 16, 4)), ("2p24", (2, 7, 16, 2)), ("2p24", (2, 2, 8, 3)), ("2p24", (2, 11, 32, 1)),
    ("2p24", (1, 4, 16, 0)),
    # several playouts per thread: each lane refills from its CTA's pool of playouts as games end
    ("2p24", (2, 11, 4, 1)), ("2p24", (2, 6, 2, 2)),
])
def test_mcts_launch_shapes_agree(dvc, variant, shape):
    """Trees per CTA, warps per CTA and chains change only who does the work."""
    kw = dict(VARIANTS[variant], playouts=8 if variant == "4p26j" else 48)
    ctx = _ctx(dvc, **kw)
    n = 11
    budgets = [40, 7, 90, 0, 33, 64, 1, 55, 20, 80, 12]
    roots = ctx.dvc_init_states(33, n)
    ref = dvc.Forest(ctx, roots, budgets, 4)
    ref.dvc_mcts_step(100)
    alt = dvc.Forest(ctx, roots, budgets, 4)
    alt.dvc_forest_tune(*shape)
    alt.dvc_mcts_step(30)
    alt.dvc_mcts_step(70)
    alt.dvc_mcts_step(64)    # budgets spent: a whole captured chunk of no-op iterations
    ctx.dvc_check()
    for t in range(n):
        assert torch.equal(ref.dvc_tree_export(t), alt.dvc_tree_export(t)), t
    assert torch.equal(ref.dvc_root_stats(), alt.dvc_root_stats())
    ocfg = oracle.OracleConfig(**kw)
    oroots = oracle.init_states(ocfg, 33, n)
    want = _oracle_trees(ocfg, oroots, 4, budgets, [2, 9])
    _check_forest(alt, alt.dvc_root_stats().cpu().numpy(), want, [2, 9])


# ---------------------------------------------------------------- ordering-aware playout policy

@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_rollout_ordered_policy_bit_exact(dvc, variant):
    kw = dict(VARIANTS[variant], policy=1)
    ocfg = oracle.OracleConfig(**kw)
    leaves = oracle.init_states(ocfg, 14, 45)
    n = len(leaves)
    tree = np.arange(n, dtype=np.uint32) * 5 + 3
    leaf = np.arange(n, dtype=np.uint32) * 11 + 1
    ctx = _ctx(dvc, **kw)
    words = torch.zeros(1, dtype=torch.int64, device="cuda")
    wins = ctx.dvc_rollout_batch(torch.from_numpy(leaves).cuda(), 37, 78, _u32(tree), _u32(leaf), words=words)
    wins = wins.cpu().numpy()
    total, differs = 0, 0
    for i in range(n):
        w, wd = oracle.rollout(ocfg, leaves[i], 37, 78, int(tree[i]), int(leaf[i]))
        assert (wins[i] == w).all(), i
        total += wd
        uniform, _ = oracle.rollout(oracle.OracleConfig(**VARIANTS[variant]), leaves[i], 37, 78, int(tree[i]),
                                    int(leaf[i]))
        differs += int((uniform != w).any())
    assert int(words.item()) == total
    assert differs > 0   # the policy does change the playouts


@pytest.mark.parametrize("variant,shape", [("2p24", (1, 0, 0, 0)), ("2p24", (2, 2, 8, 2)), ("4p26j", (1, 0, 0, 0)),
                                           ("4p26j", (2, 2, 4, 2))])
def test_mcts_ordered_policy_bit_exact(dvc, variant, shape):
    kw = dict(VARIANTS[variant], playouts=24, policy=1)
    ocfg = oracle.OracleConfig(**kw)
    n = 5
    budgets = [90, 40, 1, 70, 66]
    ctx = _ctx(dvc, **kw)
    roots = ctx.dvc_init_states(31, n)
    oroots = oracle.init_states(ocfg, 31, n)
    forest = dvc.Forest(ctx, roots, budgets, 6)
    forest.dvc_forest_tune(*shape)
    forest.dvc_mcts_step(max(budgets))
    stats = forest.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    want = _oracle_trees(ocfg, oroots, 6, budgets, range(n))
    _check_forest(forest, stats, want, range(n))


# ---------------------------------------------------------------- full game tree (Fig. 2a)

@pytest.mark.parametrize("variant,shape", [("2p24", (1, 0, 0, 0)), ("2p24", (2, 2, 8, 2)), ("4p26j", (1, 0, 0, 0)),
                                           ("4p26j", (2, 2, 4, 2))])
def test_mcts_full_tree_bit_exact(dvc, variant, shape):
    kw = dict(VARIANTS[variant], playouts=16, tree_continue=1)
    ocfg = oracle.OracleConfig(**kw)
    n = 5
    budgets = [100, 30, 1, 80, 66]
    ctx = _ctx(dvc, **kw)
    roots = ctx.dvc_init_states(35, n)
    oroots = oracle.init_states(ocfg, 35, n)
    forest = dvc.Forest(ctx, roots, budgets, 8)
    forest.dvc_forest_tune(*shape)
    forest.dvc_mcts_step(max(budgets))
    stats = forest.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    want = _oracle_trees(ocfg, oroots, 8, budgets, range(n))
    _check_forest(forest, stats, want, range(n))
    if variant == "2p24":   # with two players a correct in-tree guess is common: STOP nodes were built
        assert any((want[t][0][:, 0] == oracle.STOP).any() for t in range(n))


@pytest.mark.parametrize("variant", ["2p24", "4p26j"])
def test_rollout_from_may_stop_leaves_bit_exact(dvc, variant):
    kw = VARIANTS[variant]
    ocfg = oracle.OracleConfig(**kw)
    leaves = oracle.init_states(ocfg, 16, 40)
    leaves[::2, 22] |= 2    # every other leaf: the mover has just guessed right and may stop
    n = len(leaves)
    ids = np.arange(n, dtype=np.uint32)
    ctx = _ctx(dvc, **kw)
    words = torch.zeros(1, dtype=torch.int64, device="cuda")
    wins = ctx.dvc_rollout_batch(torch.from_numpy(leaves).cuda(), 29, 51, _u32(ids), _u32(ids), words=words)
    wins = wins.cpu().numpy()
    total = 0
    for i in range(n):
        w, wd = oracle.rollout(ocfg, leaves[i], 29, 51, i, i)
        assert (wins[i] == w).all(), i
        total += wd
    assert int(words.item()) == total


@pytest.mark.parametrize("variant,P,budgets,extra,engine", [
    ("2p24", 32, [150, 57, 1, 120], {}, 1),
    ("2p24", 32, [150, 57, 1, 120] * 40, {}, 2),
    ("4p26j", 16, [120, 64, 30], {}, 1),
    ("4p26j", 16, [120, 64, 30] * 60, {}, 2),
    ("2p24", 16, [90, 40, 77], dict(tree_continue=1), 1),
    ("3p24", 16, [90, 40, 77] * 60, dict(tree_continue=1), 2),
])
def test_forest_work_counters_match_oracle(dvc, variant, P, budgets, extra, engine):
    """Random words and game steps (one per playout guess, plus a may-stop
    leaf's first coin) counted by the GPU's playout kernels equal the
    oracle's counts for the same searches, in both engines."""
    kw = dict(VARIANTS[variant], playouts=P, **extra)
    ocfg = oracle.OracleConfig(**kw)
    n = len(budgets)
    ctx = _ctx(dvc, **kw)
    roots = ctx.dvc_init_states(31, n)
    oroots = oracle.init_states(ocfg, 31, n)
    forest = dvc.Forest(ctx, roots, budgets, 6)
    forest.dvc_forest_tune(engine)
    forest.dvc_mcts_step(max(budgets))
    work = forest.dvc_forest_work().cpu().numpy()
    ctx.dvc_check()
    out = {}

    def run(t):
        out[t] = oracle.mcts_work(ocfg, oroots[t], 6, t, int(budgets[t]))

    ths = [threading.Thread(target=run, args=(t,)) for t in range(n)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    assert int(work[0]) == sum(w for w, _ in out.values())
    assert int(work[1]) == sum(s for _, s in out.values())
    assert (forest.dvc_forest_work().cpu().numpy() == 0).all()   # read-and-zero


@pytest.mark.parametrize("variant,extra,engine", [
    ("2p24", {}, 2), ("2p24", {}, 1), ("4p26j", {}, 2), ("2p24", dict(tree_continue=1), 2),
])
def test_work_counting_off_changes_nothing_else(dvc, variant, extra, engine):
    """With work counting off (the counting-free two-player playout kernel in
    the pipeline) every tree and decision is unchanged, the counters do not
    move, and counting resumes when switched back on."""
    kw = dict(VARIANTS[variant], playouts=32, **extra)
    ctx = _ctx(dvc, **kw)
    n, budget = 600, 60
    roots = ctx.dvc_init_states(43, n)
    out = []
    for on in (True, False):
        f = dvc.Forest(ctx, roots, [budget] * n, 14)
        f.dvc_forest_tune(engine)
        f.dvc_forest_count_work(on)
        f.dvc_mcts_step(budget)
        out.append((f.dvc_root_stats().cpu().numpy(), [f.dvc_tree_export(t).cpu().numpy() for t in (0, 599)],
                    f.dvc_forest_work().cpu().numpy()))
        if not on:
            f.dvc_forest_count_work(True)
            f.dvc_forest_reset()
            f.dvc_mcts_step(budget)
            again = f.dvc_forest_work().cpu().numpy()
        f.close()
    ctx.dvc_check()
    (s0, t0, w0), (s1, t1, w1) = out
    assert (s0 == s1).all() and all((a == b).all() for a, b in zip(t0, t1))
    assert w0[0] > 0 and w0[1] > 0 and (w1 == 0).all()
    assert (again == w0).all()


@pytest.mark.parametrize("shape,receivers,donate_at", [
    ((2, 2, 16, 3), 4, 8), ((2, 2, 16, 3), 1, 31), ((2, 4, 8, 2), 2, 16), ((2, 11, 4, 1), 1, 4),
    ((2, 3, 16, 4), 15, 1),
])
def test_lane_compaction_bit_exact(dvc, shape, receivers, donate_at):
    """Lane compaction (running games handed between warps once a CTA's pool
    is empty) leaves every tree, decision and work counter unchanged; trees
    sampled against the oracle too."""
    kw = dict(VARIANTS["2p24"], playouts=64)
    ctx = _ctx(dvc, **kw)
    n, budget = 700, 70
    roots = ctx.dvc_init_states(41, n)
    out = []
    for comp in (False, True):
        f = dvc.Forest(ctx, roots, [budget] * n, 12)
        f.dvc_forest_tune(*shape)
        if comp:
            f.dvc_forest_compaction(receivers, donate_at)
        f.dvc_mcts_step(budget)
        out.append((f.dvc_root_stats().cpu().numpy(), [f.dvc_tree_export(t).cpu().numpy() for t in (0, 350, 699)],
                    f.dvc_forest_work().cpu().numpy()))
        f.close()
    ctx.dvc_check()
    (s0, t0, w0), (s1, t1, w1) = out
    assert (s0 == s1).all() and (w0 == w1).all()
    assert all((a == b).all() for a, b in zip(t0, t1))
    ocfg = oracle.OracleConfig(**kw)
    oroots = oracle.init_states(ocfg, 41, n)
    nodes, best = oracle.mcts(ocfg, oroots[350], 12, 350, budget)
    assert (t1[1][: len(nodes)] == nodes).all()


@pytest.mark.parametrize("variant,P,K,groups,extra,engine", [
    ("2p24", 32, 4, 3, {}, 1),
    ("4p26j", 16, 3, 2, {}, 2),
    ("2p24", 16, 5, 2, dict(vanilla=1), 1),
])
def test_root_parallel_merge_bit_exact(dvc, variant, P, K, groups, extra, engine):
    """Root-parallel merge (Sec. III-B): groups of K trees searched from one
    root with their own streams; the summed decision equals the oracle's
    merge of the K oracle trees."""
    kw = dict(VARIANTS[variant], playouts=P, **extra)
    ocfg = oracle.OracleConfig(**kw)
    ctx = _ctx(dvc, **kw)
    base = ctx.dvc_init_states(17, groups)
    obase = oracle.init_states(ocfg, 17, groups)
    roots = base.repeat_interleave(K, dim=0).contiguous()
    budgets = [60 + 7 * t for t in range(groups * K)]
    forest = dvc.Forest(ctx, roots, budgets, 5)
    forest.dvc_forest_tune(engine)
    forest.dvc_mcts_step(max(budgets))
    got = forest.dvc_root_merge(K).cpu().numpy()
    ctx.dvc_check()
    for g in range(groups):
        tables = [oracle.mcts(ocfg, obase[g], 5, g * K + k, budgets[g * K + k])[0] for k in range(K)]
        want = oracle.root_merge(obase[g], tables, extra.get("vanilla", 0))
        assert got[g][:4].tolist() == want.tolist(), g
        assert got[g][5] == K and got[g][6] == sum(budgets[g * K:(g + 1) * K]) and got[g][7] == 0


def test_root_merge_refuses_groups_of_other_roots(dvc):
    kw = dict(VARIANTS["2p24"], playouts=8)
    ctx = _ctx(dvc, **kw)
    roots = ctx.dvc_init_states(3, 4)               # four different roots
    forest = dvc.Forest(ctx, roots, [20] * 4, 1)
    forest.dvc_mcts_step(20)
    with pytest.raises(dvc.DvcError):
        forest.dvc_root_merge(3)                    # 3 does not divide 4: refused on the host
    forest.dvc_root_merge(2)
    with pytest.raises(dvc.DvcError) as e:
        ctx.dvc_check()                             # groups whose roots differ
    assert e.value.code == -1
