"""Host side of value-network training (no GPU): batching, shuffling and the
loss curve, with the library's train step replaced by a recorder."""
import torch

from paper_2403_10720_gb300 import value_train as vt


class _Ctx:
    def __init__(self):
        self.batches = []

    def dvc_value_train_step(self, x, y, lr, loss=None):
        self.batches.append((x[:, 0].clone(), y[:, 0].clone(), lr))
        loss.fill_(float(len(self.batches)))


def test_train_batches_are_shuffled_epochs():
    n, batch = 100, 16
    states = torch.zeros((n, 32), dtype=torch.uint8)
    states[:, 0] = torch.arange(n, dtype=torch.uint8)
    labels = torch.zeros((n, 4))
    labels[:, 0] = torch.arange(n, dtype=torch.float32)
    ctx = _Ctx()
    curve = vt.train(ctx, states, labels, epochs=3, batch=batch, lr=0.5, seed=4)
    per_epoch = n // batch                       # the last partial batch of an epoch is dropped
    assert len(ctx.batches) == 3 * per_epoch and len(curve) == 3
    for e in range(3):
        rows = torch.cat([x for x, _, _ in ctx.batches[e * per_epoch:(e + 1) * per_epoch]])
        assert len(set(rows.tolist())) == per_epoch * batch      # no row twice within an epoch
    for x, y, lr in ctx.batches:
        assert torch.equal(x.float(), y) and lr == 0.5           # states and labels stay paired
    assert curve[0] == sum(range(1, per_epoch + 1)) / per_epoch   # mean of the epoch's step losses
    again = _Ctx()
    vt.train(again, states, labels, epochs=3, batch=batch, lr=0.5, seed=4)
    assert all(torch.equal(a[0], b[0]) for a, b in zip(ctx.batches, again.batches))   # seeded


def test_mean_abs_error_counts_seats_in_play():
    states = torch.zeros((2, 32), dtype=torch.uint8)
    states[0, 26], states[1, 26] = 2, 4
    pred = torch.tensor([[0.5, 0.5, 9.0, 9.0], [0.25, 0.25, 0.25, 0.25]])
    labels = torch.tensor([[1.0, 0.0, 0.0, 0.0], [0.25, 0.25, 0.25, 0.25]])
    assert abs(vt.mean_abs_error(pred, labels, states) - 1.0 / 6.0) < 1e-7
