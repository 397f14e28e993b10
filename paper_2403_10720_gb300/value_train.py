"""Training and evaluation of the value network through the C ABI.

Labels are rollout estimates: each state's win probabilities are the win
fractions of `playouts` random playouts from it (dvc_rollout_batch).  All
arithmetic runs in libdvc; this module only chooses batches.
"""
import time

import numpy as np
import torch


def label_states(ctx, states, playouts=1024, seed=0x5EED, chunk=16384):
    """Win fractions per absolute seat (n x 4 FP32) from `playouts` playouts."""
    n = states.shape[0]
    labels = torch.empty((n, 4), dtype=torch.float32, device=states.device)
    ids = torch.arange(n, dtype=torch.int32, device=states.device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        wins = ctx.dvc_rollout_batch(states[a:b], playouts, seed, ids[a:b], ids[a:b])
        labels[a:b] = wins.float() / playouts
    return labels


def make_dataset(ctx, n, root_seed, playouts=1024, seed=0x5EED):
    states = ctx.dvc_init_states(root_seed, n)
    return states, label_states(ctx, states, playouts, seed)


def train(ctx, states, labels, epochs=8, batch=8192, lr=1e-3, seed=0):
    """Shuffled mini-batch AdamW; returns the mean loss of each epoch."""
    g = torch.Generator(device=states.device).manual_seed(seed)
    n = states.shape[0]
    loss = torch.zeros(1, device=states.device)
    curve = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g, device=states.device)
        tot, cnt = 0.0, 0
        for a in range(0, n - batch + 1, batch):
            idx = perm[a:a + batch]
            ctx.dvc_value_train_step(states[idx].contiguous(), labels[idx].contiguous(), lr, loss=loss)
            tot += loss.item()
            cnt += 1
        curve.append(tot / max(cnt, 1))
    return curve


def mean_abs_error(pred, labels, states):
    """Mean |p - label| over the seats in play."""
    nplayers = states[:, 26].long()
    mask = torch.arange(4, device=pred.device)[None, :] < nplayers[:, None]
    return float(((pred - labels).abs() * mask).sum() / mask.sum())


def rollout_estimate(ctx, states, k, seed=0xE57):
    ids = torch.arange(states.shape[0], dtype=torch.int32, device=states.device)
    return ctx.dvc_rollout_batch(states, k, seed, ids, ids).float() / k


def timed(fn, reps=5):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps
