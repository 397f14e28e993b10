"""Host-side scheduling of a forest's search (no GPU): where the tail of long
budgets starts, and the engine switch around it."""
import numpy as np

from paper_2403_10720_gb300 import autotune


def test_tail_start_leaves_at_most_the_threshold_running():
    rng = np.random.default_rng(3)
    b = np.floor(np.exp(rng.uniform(np.log(1000), np.log(100000), size=16384))).astype(np.int32)
    for per_sm in (5, 12, 16):
        cut = autotune.tail_start(b, 152, per_sm)
        assert (b > cut).sum() <= per_sm * 152 < (b >= cut).sum() + per_sm * 152
        assert 0 < cut < b.max()


def test_tail_start_edge_cases():
    assert autotune.tail_start([5] * 10, 152) == 0           # few trees: the tail is the whole search
    assert autotune.tail_start([100] * 5000, 152) is None    # equal budgets: no tail
    assert autotune.tail_start([1, 2, 3, 4], 1, per_sm=2) == 2


class _Forest:
    def __init__(self):
        self.calls = []

    def dvc_forest_tune(self, *shape):
        self.calls.append(("tune", shape))

    def dvc_forest_order(self, order, n_active=0):
        self.calls.append(("order", None if order is None else [int(t) for t in order], n_active))

    def dvc_mcts_step(self, n):
        self.calls.append(("step", n))


def test_step_with_tail_splits_the_iterations():
    f = _Forest()
    b = [10, 20, 30, 40, 50]
    autotune.step_with_tail(f, b, (2, 1, 1, 8), sms=1, pack_per_sm=3, tail_per_sm=1)
    # 3 trees left after iteration 20 (packed fused shape), 1 after 40 (one tree per CTA); each
    # fused chunk first lists the running trees, longest remaining budget first
    assert f.calls == [("tune", (2, 1, 1, 8)), ("step", 20),
                       ("tune", autotune.PACK_SHAPE), ("order", [4, 3, 2, 0, 1], 3), ("step", 20),
                       ("tune", autotune.TAIL_SHAPE), ("order", [4, 0, 1, 2, 3], 1), ("step", 10),
                       ("order", None, 0)]
    g = _Forest()
    autotune.step_with_tail(g, [7] * 8, (2, 1, 1, 8), sms=1, pack_per_sm=2, tail_per_sm=1)
    assert g.calls == [("tune", (2, 1, 1, 8)), ("step", 7)]


def test_packed_chunks_keep_finished_trees_out():
    f = _Forest()
    b = np.array([5000, 1000, 3000, 2500])
    autotune._packed_steps(f, b, 0, 5000, chunk=2000)
    steps = [c for c in f.calls if c[0] == "step"]
    orders = [c for c in f.calls if c[0] == "order"]
    assert [c[1] for c in steps] == [2000, 2000, 1000]
    assert orders[0][1:] == ([0, 2, 3, 1], 4)                # all running, longest first
    assert orders[1][1:] == ([0, 2, 3, 1], 3)                # tree 1 ended at 1000
    assert orders[2][1:] == ([0, 1, 2, 3], 1)                # only tree 0 is left
