"""Self-play between two leaf evaluators, and move agreement.

Games follow the model the tree searches (Sec. III-A): the seat to move
draws, makes one guess chosen by a UCT search from its own view, and the turn
passes.  Every move of every live game is a query to a dvc_server (searches of
all games run together on the device); the decisions are applied to the true
states with dvc_play_move.  In game g the value-network agent plays seat
g mod P and the playout agent the other seats, so each agent moves first in
its share of the games.  All arithmetic runs in libdvc; this module only
schedules queries and counts.
"""
import math
import time

import numpy as np
import torch

from . import DVC_MODE_ROLLOUT, DVC_MODE_VALUE


def play_games(ctx, server, n_games, budget, root_seed, seed, value_budget=None, max_turns=400, poll_iters=256):
    """Play n_games fresh deals (dvc_init_states(root_seed, n_games)) to the
    end.  Returns a dict: winners (n,), value_seat (n,), turns, decisions,
    wall seconds, and the value agent's win rate with a 95% interval."""
    value_budget = budget if value_budget is None else value_budget
    states = ctx.dvc_init_states(root_seed, n_games)
    nplayers = int(states[0, 26].item())
    value_seat = np.arange(n_games) % nplayers
    game_ids = torch.arange(n_games, dtype=torch.int32, device=states.device)
    actions = torch.empty(n_games, dtype=torch.int32, device=states.device)
    decisions = {DVC_MODE_ROLLOUT: 0, DVC_MODE_VALUE: 0}
    t0 = time.perf_counter()
    turn = 0
    while turn < max_turns:
        h = states.cpu().numpy()
        live = np.nonzero(h[:, 28] == 0xFF)[0]
        if len(live) == 0:
            break
        act = np.full(n_games, -1, dtype=np.int32)
        for g in live:
            mode = DVC_MODE_VALUE if h[g, 23] == value_seat[g] else DVC_MODE_ROLLOUT
            server.dvc_server_submit(h[g], value_budget if mode == DVC_MODE_VALUE else budget, mode,
                                     turn * n_games + int(g))
            decisions[mode] += 1
        got = 0
        while got < len(live):
            for r in server.dvc_server_poll(poll_iters):
                act[int(r["query_id"]) % n_games] = r["best_action"]
                got += 1
        actions.copy_(torch.from_numpy(act))
        ctx.dvc_play_move(states, actions, seed, turn, game_ids)
        turn += 1
    ctx.dvc_check()
    wall = time.perf_counter() - t0
    h = states.cpu().numpy()
    winners = h[:, 28].astype(np.int64)
    done = winners != 0xFF
    wins = int((winners[done] == value_seat[done]).sum())
    n_done = int(done.sum())
    rate = wins / max(n_done, 1)
    half = 1.96 * math.sqrt(max(rate * (1 - rate), 1e-12) / max(n_done, 1))
    return {
        "winners": winners, "value_seat": value_seat, "turns": turn, "games_finished": n_done,
        "value_wins": wins, "value_win_rate": rate, "ci95": [rate - half, rate + half],
        "fair_share": 1.0 / nplayers, "decisions": {"rollout": decisions[DVC_MODE_ROLLOUT],
                                                     "value": decisions[DVC_MODE_VALUE]},
        "wall_s": wall, "decisions_per_s": (decisions[0] + decisions[1]) / wall,
    }


def decide(ctx, dvc, roots, budget, mode, seed, tree_ids=None):
    """Best action of a UCT search (one tree per root) in the given leaf mode."""
    forest = dvc.Forest(ctx, roots, [budget] * roots.shape[0], seed, tree_ids=tree_ids)
    forest.dvc_mcts_step(budget, mode=mode)
    best = forest.dvc_root_stats()[:, 0].clone()
    forest.close()
    return best


def move_agreement(ctx, dvc, roots, budget, strong_budget, seed):
    """Decisions of the value agent and the playout agent at `budget`, each
    compared with a strong playout search (strong_budget iterations) and with
    each other, on the same roots.  Returns fractions."""
    v = decide(ctx, dvc, roots, budget, DVC_MODE_VALUE, seed)
    r = decide(ctx, dvc, roots, budget, DVC_MODE_ROLLOUT, seed)
    s = decide(ctx, dvc, roots, strong_budget, DVC_MODE_ROLLOUT, seed + 1)
    ctx.dvc_check()
    f = lambda a, b: float((a == b).float().mean())  # noqa: E731
    return {"value_vs_strong": f(v, s), "rollout_vs_strong": f(r, s), "value_vs_rollout": f(v, r),
            "positions": int(roots.shape[0]), "budget": budget, "strong_budget": strong_budget}
