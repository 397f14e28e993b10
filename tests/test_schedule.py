"""Host-side scheduling of a forest's search (no GPU): where the tail of long
budgets starts, and the engine switch around it."""
import numpy as np

from paper_2403_10720_gb300 import autotune


def test_tail_start_leaves_at_most_the_threshold_running():
    rng = np.random.default_rng(3)
    b = np.floor(np.exp(rng.uniform(np.log(1000), np.log(100000), size=16384))).astype(np.int32)
    cut = autotune.tail_start(b, 152)
    assert (b > cut).sum() <= 12 * 152 < (b >= cut).sum() + 12 * 152
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

    def dvc_mcts_step(self, n):
        self.calls.append(("step", n))


def test_step_with_tail_splits_the_iterations():
    f = _Forest()
    autotune.step_with_tail(f, [10, 20, 30, 40, 50], (2, 1, 1, 8), sms=1, per_sm=2)
    # 2 trees left after iteration 30: tuned shape for 30 iterations, then the tail shape for 20
    assert f.calls == [("tune", (2, 1, 1, 8)), ("step", 30), ("tune", autotune.TAIL_SHAPE), ("step", 20)]
    g = _Forest()
    autotune.step_with_tail(g, [7] * 8, (2, 1, 1, 8), sms=1, per_sm=2)
    assert g.calls == [("tune", (2, 1, 1, 8)), ("step", 7)]
