"""Host scheduling of forest-based games (no GPU): who searches which game,
how searches are keyed, and how decisions reach the game and are counted.
The library is replaced by fakes that record the calls."""
import numpy as np
import torch

import paper_2403_10720_gb300 as dvc
from paper_2403_10720_gb300 import selfplay


class _Game:
    """Two-player games; seat `cur` alternates each turn; game g ends after
    3 + g % 4 moves with the player to move as winner."""

    def __init__(self):
        self.moves = []

    def dvc_init_states(self, seed, n):
        s = torch.zeros((n, 32), dtype=torch.uint8)
        s[:, 26] = 2
        s[:, 28] = 0xFF
        s[:, 23] = torch.arange(n) % 2          # game g starts with seat g mod 2
        return s

    def dvc_play_move(self, states, actions, seed, turn, game_ids):
        a = actions.numpy().copy()
        self.moves.append((turn, a))
        for g in range(states.shape[0]):
            if states[g, 28] != 0xFF:
                assert a[g] == -1
                continue
            assert a[g] == turn * states.shape[0] + g  # the decision of this game's search
            if turn + 1 >= 3 + g % 4:
                states[g, 28] = states[g, 23]
            else:
                states[g, 23] ^= 1

    def dvc_check(self):
        pass


class _Forest:
    made = []

    def __init__(self, ctx, roots, budgets, seed, tree_ids=None):
        self.ctx, self.n, self.ids = ctx, roots.shape[0], np.asarray(tree_ids)
        _Forest.made.append((ctx, self.n, list(budgets), seed, self.ids.copy(), roots[:, 23].clone()))

    def dvc_mcts_step(self, n):
        pass

    def dvc_root_stats(self):
        out = torch.zeros((self.n, 8), dtype=torch.int32)
        out[:, 0] = torch.from_numpy(self.ids.astype(np.int32))   # "best action" = the tree id, to trace routing
        return out

    def close(self):
        pass


def test_forest_agents_route_and_count(monkeypatch):
    monkeypatch.setattr(dvc, "Forest", _Forest)
    _Forest.made.clear()
    game = _Game()
    a, b = object(), object()
    n = 8
    out = selfplay.play_forest_agents(game, (a, 5), (b, 7), n, root_seed=1, seed=9)
    assert out["games_finished"] == n and out["turns"] == 6    # the longest game lasts 3 + 3 moves
    # agent A plays seat g mod 2 of game g: every forest of A holds only positions where that seat moves
    a_seat = np.arange(n) % 2
    for ctx, cnt, budgets, seed, ids, movers in _Forest.made:
        games = ids % n
        assert seed == 9 and budgets == [5 if ctx is a else 7] * cnt
        want = a_seat[games] if ctx is a else 1 - a_seat[games]
        assert (movers.numpy() == want).all()
    # every live game got exactly one decision per turn
    assert out["decisions_a"] + out["decisions_b"] == sum(3 + g % 4 for g in range(n))
    # game g starts with seat g mod 2 = A's seat; the winner is the player to move at its last move
    for g in range(n):
        moves = 3 + g % 4
        winner = (g % 2) ^ ((moves - 1) % 2)
        assert out["winners"][g] == winner
    assert out["a_wins"] == sum(int(out["winners"][g] == a_seat[g]) for g in range(n))


class _Server:
    def __init__(self):
        self.queue, self.submitted = [], []

    def dvc_server_submit(self, root, budget, mode, qid):
        self.submitted.append((int(root[23]), budget, mode, qid))
        self.queue.append(qid)

    def dvc_server_poll(self, iters):
        out = [{"query_id": q, "best_action": q} for q in self.queue[:3]]   # a few results per poll
        self.queue = self.queue[3:]
        return out


def test_server_agents_route_and_count():
    game = _Game()
    sa, sb = _Server(), _Server()
    n = 8
    out = selfplay.play_agents(game, (sa, dvc.DVC_MODE_VALUE, 5), (sb, dvc.DVC_MODE_ROLLOUT, 7), n, root_seed=1,
                               seed=9)
    a_seat = np.arange(n) % 2
    for srv, mode, budget, seat_of in ((sa, dvc.DVC_MODE_VALUE, 5, lambda g: a_seat[g]),
                                       (sb, dvc.DVC_MODE_ROLLOUT, 7, lambda g: 1 - a_seat[g])):
        assert srv.submitted
        for mover, b, m, qid in srv.submitted:
            assert m == mode and b == budget and mover == seat_of(qid % n)
    assert out["decisions_a"] == len(sa.submitted) and out["decisions_b"] == len(sb.submitted)
    assert out["games_finished"] == n and out["turns"] == 6
