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
