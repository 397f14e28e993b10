"""Self-play between two search agents, and move agreement.

Games follow the model the tree searches (Sec. III-A): the seat to move
draws, makes one guess chosen by a UCT search from its own view, and the turn
passes.  Every move of every live game is a query to a dvc_server (searches of
all games run together on the device), or, for agents a server does not hold
(vanilla MCTS-dvc), one tree of a per-turn forest; the decisions are applied to the true
states with dvc_play_move.  In game g agent A plays seat g mod P and agent B
the other seats, so each agent moves first in its share of the games.  An
agent is a server (its context fixes the playout policy) with a leaf mode and
an iteration budget: the value-network agent against the playout agent, or
the ordering-aware playout policy against the uniform one.  All arithmetic
runs in libdvc; this module only schedules queries and counts.
"""
import math
import time

import numpy as np
import torch

from . import DVC_MODE_ROLLOUT, DVC_MODE_VALUE


def play_games(ctx, server, n_games, budget, root_seed, seed, value_budget=None, max_turns=400, poll_iters=256):
    """The value-network agent against the playout agent, both searching
    through `server`.  Returns play_agents' dict with the value agent as
    agent A ("value_*" keys as aliases)."""
    value_budget = budget if value_budget is None else value_budget
    out = play_agents(ctx, (server, DVC_MODE_VALUE, value_budget), (server, DVC_MODE_ROLLOUT, budget), n_games,
                      root_seed, seed, max_turns, poll_iters)
    out["value_seat"] = out["a_seat"]
    out["value_wins"] = out["a_wins"]
    out["value_win_rate"] = out["a_win_rate"]
    out["decisions"] = {"value": out["decisions_a"], "rollout": out["decisions_b"]}
    return out


def play_agents(ctx, agent_a, agent_b, n_games, root_seed, seed, max_turns=400, poll_iters=256):
    """Play n_games fresh deals (dvc_init_states(root_seed, n_games) of ctx)
    to the end between agent A (seat g mod P of game g) and agent B (the other
    seats).  An agent is (server, mode, budget): its moves are queries to that
    server.  Returns a dict: winners (n,), a_seat (n,), turns, decisions per
    agent, wall seconds, and agent A's win rate with a 95% interval."""
    states = ctx.dvc_init_states(root_seed, n_games)
    nplayers = int(states[0, 26].item())
    a_seat = np.arange(n_games) % nplayers
    game_ids = torch.arange(n_games, dtype=torch.int32, device=states.device)
    actions = torch.empty(n_games, dtype=torch.int32, device=states.device)
    decisions = [0, 0]
    servers = [agent_a[0]] if agent_a[0] is agent_b[0] else [agent_a[0], agent_b[0]]
    t0 = time.perf_counter()
    turn = 0
    while turn < max_turns:
        h = states.cpu().numpy()
        live = np.nonzero(h[:, 28] == 0xFF)[0]
        if len(live) == 0:
            break
        act = np.full(n_games, -1, dtype=np.int32)
        for g in live:
            who = 0 if h[g, 23] == a_seat[g] else 1
            server, mode, budget = agent_a if who == 0 else agent_b
            server.dvc_server_submit(h[g], budget, mode, turn * n_games + int(g))
            decisions[who] += 1
        got = 0
        while got < len(live):
            for sv in servers:
                for r in sv.dvc_server_poll(poll_iters):
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
    wins = int((winners[done] == a_seat[done]).sum())
    n_done = int(done.sum())
    rate = wins / max(n_done, 1)
    half = 1.96 * math.sqrt(max(rate * (1 - rate), 1e-12) / max(n_done, 1))
    return {
        "winners": winners, "a_seat": a_seat, "turns": turn, "games_finished": n_done,
        "a_wins": wins, "a_win_rate": rate, "ci95": [rate - half, rate + half],
        "fair_share": 1.0 / nplayers, "decisions_a": decisions[0], "decisions_b": decisions[1],
        "wall_s": wall, "decisions_per_s": (decisions[0] + decisions[1]) / wall,
    }


def play_forest_agents(game, agent_a, agent_b, n_games, root_seed, seed, max_turns=400):
    """play_agents for agents a server does not hold (vanilla trees): each
    turn, every agent searches all positions where it is to move as one
    forest.  An agent is (ctx, budget): its context fixes the tree and the
    playout policy.  The search of game g at turn k is keyed by tree id
    k * n_games + g.  Same return dict as play_agents."""
    from . import Forest
    states = game.dvc_init_states(root_seed, n_games)
    nplayers = int(states[0, 26].item())
    a_seat = np.arange(n_games) % nplayers
    game_ids = torch.arange(n_games, dtype=torch.int32, device=states.device)
    actions = torch.empty(n_games, dtype=torch.int32, device=states.device)
    decisions = [0, 0]
    t0 = time.perf_counter()
    turn = 0
    while turn < max_turns:
        h = states.cpu().numpy()
        live = np.nonzero(h[:, 28] == 0xFF)[0]
        if len(live) == 0:
            break
        act = np.full(n_games, -1, dtype=np.int32)
        for who, (ctx, budget) in enumerate((agent_a, agent_b)):
            mine = live[(h[live, 23] == a_seat[live]) == (who == 0)]
            if len(mine) == 0:
                continue
            roots = states[torch.from_numpy(mine).to(states.device)].contiguous()
            forest = Forest(ctx, roots, [budget] * len(mine), seed, tree_ids=turn * n_games + mine)
            forest.dvc_mcts_step(budget)
            act[mine] = forest.dvc_root_stats()[:, 0].cpu().numpy()
            forest.close()
            decisions[who] += len(mine)
        actions.copy_(torch.from_numpy(act))
        game.dvc_play_move(states, actions, seed, turn, game_ids)
        turn += 1
    game.dvc_check()
    wall = time.perf_counter() - t0
    h = states.cpu().numpy()
    winners = h[:, 28].astype(np.int64)
    done = winners != 0xFF
    wins = int((winners[done] == a_seat[done]).sum())
    n_done = int(done.sum())
    rate = wins / max(n_done, 1)
    half = 1.96 * math.sqrt(max(rate * (1 - rate), 1e-12) / max(n_done, 1))
    return {
        "winners": winners, "a_seat": a_seat, "turns": turn, "games_finished": n_done,
        "a_wins": wins, "a_win_rate": rate, "ci95": [rate - half, rate + half],
        "fair_share": 1.0 / nplayers, "decisions_a": decisions[0], "decisions_b": decisions[1],
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
