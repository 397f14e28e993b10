"""Self-play moves (dvc_play_move) against the oracle, and games between the
value-network agent and the playout agent played through the server."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

VARIANTS = {
    "2p24": dict(nplayers=2, ntiles=24, deal=4, max_predraw=0, max_revealed=5),
    "3p24": dict(nplayers=3, ntiles=24, deal=4, max_predraw=6, max_revealed=3),
    "4p26j": dict(nplayers=4, ntiles=26, deal=3, max_predraw=8, max_revealed=3),
}


@pytest.fixture(scope="module")
def dvc():
    import paper_2403_10720_gb300 as m
    from paper_2403_10720_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_play_move_bit_exact(dvc, variant):
    """Random legal guesses (and some skipped moves) applied turn by turn to
    300 games: every record equals the oracle's after every turn."""
    kw = VARIANTS[variant]
    ctx = dvc.Context(dvc.Config(**kw), 0)
    n, seed = 300, 0xABCDEF0123
    states = ctx.dvc_init_states(41, n)
    want = oracle.init_states(oracle.OracleConfig(**kw), 41, n)
    assert (states.cpu().numpy() == want).all()
    game_ids = torch.from_numpy((np.arange(n, dtype=np.uint32) * 7 + 3).view(np.int32)).cuda()
    rng = np.random.default_rng(5)
    for turn in range(60):
        act = np.full(n, -1, dtype=np.int32)
        for g in range(n):
            if want[g][28] != 0xFF or rng.random() < 0.05:
                continue
            legal = oracle.legal_actions(want[g])
            act[g] = legal[rng.integers(len(legal))]
        ctx.dvc_play_move(states, torch.from_numpy(act).cuda(), seed, turn, game_ids)
        for g in range(n):
            if act[g] >= 0:
                rc, want[g] = oracle.play_move(want[g], int(act[g]), seed, g * 7 + 3, turn)
                assert rc == 0
        got = states.cpu().numpy()
        ctx.dvc_check()
        assert (got == want).all(), (turn, np.nonzero((got != want).any(1))[0][:5])
        if (want[:, 28] != 0xFF).all():
            break
    assert (want[:, 28] != 0xFF).mean() > 0.5   # most games played to the end


def test_play_move_rejects_illegal_guess(dvc):
    ctx = dvc.Context(dvc.Config(**VARIANTS["2p24"]), 0)
    states = ctx.dvc_init_states(3, 4)
    before = states.clone()
    h = states.cpu().numpy()
    act = np.array([oracle.legal_actions(h[g])[0] for g in range(4)], dtype=np.int32)
    cur = int(h[1][23])
    act[1] = (cur << 10) | 0   # a guess at the mover's own row
    ctx.dvc_play_move(states, torch.from_numpy(act).cuda(), 1, 0)
    with pytest.raises(dvc.DvcError) as err:
        ctx.dvc_check()
    assert err.value.code == -1   # DVC_E_INVALID
    assert torch.equal(states[1], before[1])
    for g in (0, 2, 3):
        assert (states[g].cpu().numpy() == oracle.play_move(h[g], int(act[g]), 1, g, 0)[1]).all()


def _direct(dvc, ctx, root, budget, qid, seed, mode):
    f = dvc.Forest(ctx, torch.from_numpy(root[None]).cuda(), [budget], seed, tree_ids=[qid])
    f.dvc_mcts_step(budget, mode)
    a = int(f.dvc_root_stats().cpu().numpy()[0][0])
    f.close()
    return a


def test_selfplay_games_end_and_repeat(dvc):
    """Sixteen games between the (untrained) value agent and the playout agent
    end with a winner, replay identically, and each first move is the decision
    the same search makes alone."""
    from paper_2403_10720_gb300 import selfplay
    kw = dict(VARIANTS["2p24"], playouts=16)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    ctx.dvc_value_init(4)
    runs = []
    for _ in range(2):
        server = dvc.Server(ctx, 1 << 28, 64, value_share_pct=50, seed=12)
        runs.append(selfplay.play_games(ctx, server, 16, 48, root_seed=8, seed=21, poll_iters=32))
        server.close()
    a, b = runs
    assert a["games_finished"] == 16 and (a["winners"] < 2).all()
    assert (a["winners"] == b["winners"]).all() and a["turns"] == b["turns"]
    assert a["decisions"]["value"] > 0 and a["decisions"]["rollout"] > 0
    roots = ctx.dvc_init_states(8, 16).cpu().numpy()
    server = dvc.Server(ctx, 1 << 28, 64, value_share_pct=50, seed=12)
    for g in range(4):
        mode = 1 if roots[g][23] == g % 2 else 0
        server.dvc_server_submit(roots[g], 48, mode, g)
    got = {}
    while len(got) < 4:
        for r in server.dvc_server_poll(32):
            got[r["query_id"]] = r["best_action"]
    for g in range(4):
        mode = 1 if roots[g][23] == g % 2 else 0
        assert got[g] == _direct(dvc, ctx, roots[g], 48, g, 12, mode), g


def test_move_agreement_fractions(dvc):
    from paper_2403_10720_gb300 import selfplay
    kw = dict(VARIANTS["2p24"], max_predraw=10, playouts=16)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    ctx.dvc_value_init(4)
    roots = ctx.dvc_init_states(19, 64)
    ag = selfplay.move_agreement(ctx, dvc, roots, 32, 256, seed=3)
    for k in ("value_vs_strong", "rollout_vs_strong", "value_vs_rollout"):
        assert 0.0 <= ag[k] <= 1.0
    assert ag["positions"] == 64


@pytest.mark.parametrize("variant", ["2p24", "4p26j"])
def test_play_move_full_game_bit_exact(dvc, variant):
    """The full game (Fig. 2a): a correct guess keeps the turn and STOP passes
    it; random actions, STOP included when allowed, match the oracle."""
    kw = dict(VARIANTS[variant], tree_continue=1)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    n, seed = 200, 0x51
    states = ctx.dvc_init_states(43, n)
    want = oracle.init_states(oracle.OracleConfig(**kw), 43, n)
    rng = np.random.default_rng(9)
    stops = 0
    for turn in range(120):
        act = np.full(n, -1, dtype=np.int32)
        for g in range(n):
            if want[g][28] != 0xFF:
                continue
            legal = oracle.legal_actions(want[g]).tolist()
            if want[g][22] & 2:
                legal.append(oracle.STOP)
            act[g] = legal[rng.integers(len(legal))]
            stops += int(act[g] == oracle.STOP)
        ctx.dvc_play_move(states, torch.from_numpy(act).cuda(), seed, turn)
        for g in range(n):
            if act[g] >= 0:
                rc, want[g] = oracle.play_move(want[g], int(act[g]), seed, g, turn, cont=1)
                assert rc == 0
        ctx.dvc_check()
        assert (states.cpu().numpy() == want).all(), turn
        if (want[:, 28] != 0xFF).all():
            break
    assert stops > 0
