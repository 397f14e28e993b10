"""Host side of the Poisson serving driver (no GPU): every query is
submitted once, in arrival order, and its latency is taken from the
server's own submit/done stamps."""
import numpy as np

from paper_2403_10720_gb300 import serving


class _Server:
    """Finishes a query `budget` polls after it was submitted; stamps in
    seconds of a fake clock advanced by one per poll."""

    def __init__(self):
        self.clock = 0.0
        self.pending, self.order = [], []

    def dvc_server_submit(self, root, budget, mode, qid):
        self.order.append(qid)
        self.pending.append([qid, budget, self.clock])

    def dvc_server_poll(self, iters):
        self.clock += 1.0
        out, keep = [], []
        for q in self.pending:
            q[1] -= 1
            if q[1] <= 0:
                out.append({"query_id": q[0], "t_submit": q[2], "t_done": self.clock, "best_action": 0})
            else:
                keep.append(q)
        self.pending = keep
        return out

    def dvc_server_stats(self):
        return {"resident": len(self.pending)}


def test_poisson_run_submits_every_query_once_in_order():
    srv = _Server()
    n = 50
    roots = np.zeros((n, 32), dtype=np.uint8)
    budgets = np.arange(n) % 5 + 1
    out = serving.poisson_run(srv, roots, budgets, np.zeros(n, dtype=int), rate=1e6, seed=3)
    assert srv.order == list(range(n))
    assert out["queries"] == n and len(out["results"]) == n
    lat = sorted(float(b) for b in budgets)           # a query takes exactly its budget in polls
    assert abs(out["p50_ms"] - 1e3 * np.percentile(lat, 50)) < 1e-6
    assert abs(out["p99_ms"] - 1e3 * np.percentile(lat, 99)) < 1e-6


class _Ctx:
    """A variant's context: roots tagged with the variant and a deal number;
    a move bumps byte 30 (a move counter) and ends the game at 3 moves."""

    def __init__(self, v, nplayers, ntiles):
        import types
        self.v = v
        self.cfg = types.SimpleNamespace(nplayers=nplayers, ntiles=ntiles)
        self.deals = 0

    def dvc_init_states(self, seed, n):
        import torch
        s = torch.zeros((n, 32), dtype=torch.uint8)
        s[:, 26] = self.cfg.nplayers
        s[:, 27] = self.cfg.ntiles
        s[:, 28] = 0xFF
        s[:, 29] = self.v
        self.deals += n
        return s

    def dvc_play_move(self, st, acts, seed, turn, ids, stream=None):
        assert (st[:, 29] == self.v).all()           # each game's moves go to its own variant
        st[:, 30] += 1
        st[st[:, 30] >= 3, 28] = 0
        return st


def test_game_serving_run_routes_moves_and_redeals():
    srv = _Server()
    ctxs = [_Ctx(0, 2, 24), _Ctx(1, 4, 26), _Ctx(2, 3, 24)]
    out = serving.game_serving_run(srv, ctxs, n_games=30, rate=1e5, duration_s=0.05, budget_lo=1, budget_hi=4,
                                   value_frac=0.5, seed=2, device="cpu")
    assert out["queries"] == len(srv.order) and out["queries"] > 0
    assert out["moves_played"] == out["queries"]
    # every re-deal takes exactly three moves of one game; at most two moves
    # per game are not yet followed by one
    assert 3 * out["games_redealt"] <= out["moves_played"] <= 3 * out["games_redealt"] + 2 * 30
    assert sorted(out["by_variant"]) == ["2p24", "3p24", "4p26"]
    assert sum(v["queries"] for v in out["by_variant"].values()) == out["queries"]
    assert sum(v["queries"] for v in out["by_mode"].values()) == out["queries"]
    if out["queries"] >= 90:
        assert out["games_redealt"] > 0
