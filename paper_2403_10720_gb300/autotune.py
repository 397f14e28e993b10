"""Launch-shape autotuner for dvc_mcts_step.

Times every candidate (engine, trees per CTA, warps per CTA, chains) on a
budget-scaled copy of the forest -- the same roots and seed, budgets scaled
down so a trial takes a fraction of a second -- with CUDA events, and keeps the
fastest.  Results are identical for every shape (the library guarantees it),
so only time is compared.  Choices are cached per workload signature and GPU in
~/.cache/dvc/autotune.json.
"""
import json
import os

import numpy as np
import torch

# The last five give each rollout CTA exactly one warp per 32 playouts of its
# trees: with few playouts per leaf and uneven budgets, idle warps would hold
# registers until the CTA's longest game ends.
CANDIDATES = [(2, 0, 0, 0), (2, 2, 16, 8), (2, 4, 16, 4), (2, 4, 16, 8), (2, 2, 8, 8), (2, 0, 32, 2), (1, 0, 16, 0),
              (1, 0, 32, 0), (2, 1, 1, 16), (2, 1, 1, 8), (2, 2, 2, 8), (2, 2, 2, 16), (2, 4, 4, 8)]
_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "dvc", "autotune.json")


def _signature(cfg, n, budgets):
    b = np.asarray(budgets)
    name = torch.cuda.get_device_name()
    return (f"{name}|p{cfg.nplayers}t{cfg.ntiles}po{cfg.playouts}|n{n}|"
            f"b{int(b.min())}-{int(np.median(b))}-{int(b.max())}")


def _load():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    try:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as f:
            json.dump(d, f, indent=1)
    except OSError:
        pass


def tune(dvc, ctx, roots, budgets, seed, scale=0.05, candidates=None, use_cache=True, verbose=False):
    """Returns the fastest (engine, trees_per_cta, warps_per_cta, chains)."""
    budgets = np.asarray(budgets, dtype=np.int32)
    key = _signature(ctx.cfg, len(budgets), budgets)
    cache = _load() if use_cache else {}
    if key in cache:
        return tuple(cache[key])
    small = np.maximum(1, (budgets * scale).astype(np.int32))
    f = dvc.Forest(ctx, roots, small, seed)
    best, best_ms, trials = None, float("inf"), []
    for cand in candidates or CANDIDATES:
        try:
            f.dvc_forest_tune(*cand)
        except Exception:
            continue
        times = []
        for _ in range(2):
            f.dvc_forest_reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f.dvc_mcts_step(int(small.max()))
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        ms = min(times)
        trials.append((cand, ms))
        if ms < best_ms:
            best, best_ms = cand, ms
    f.close()
    if verbose:
        for c, ms in trials:
            print(f"autotune {c}: {ms:.2f} ms")
    if use_cache and best is not None:
        cache[key] = list(best)
        _save(cache)
    return best


# The tail of an uneven forest, measured on four-player forests in chunks of
# 2,000 iterations (budgets 1k-100k): with at most 16 running trees per SM the
# fused engine with 4 trees x 4 warps per CTA, its CTAs filled with running
# trees of similar remaining budgets, beats the pipeline (76 against 90 us per
# iteration with 2,438 trees left, 64 against 85 with 1,785); with at most 5
# per SM one tree per CTA is fastest (52 against 55 us with 770 left).  Without
# the repacking, CTAs of several trees keep their finished trees' warps and
# lose to one tree per CTA.
PACK_TREES_PER_SM = 16
PACK_SHAPE = (1, 4, 4, 0)
TAIL_TREES_PER_SM = 5
TAIL_SHAPE = (1, 1, 1, 0)
PACK_CHUNK = 2000


def tail_start(budgets, sms, per_sm=TAIL_TREES_PER_SM):
    """First iteration at which at most per_sm * sms trees of a fresh forest
    with these budgets are still running (None if that never happens before
    the longest budget ends)."""
    b = np.sort(np.asarray(budgets, dtype=np.int64))[::-1]
    k = per_sm * sms
    if k >= len(b):
        return 0
    return int(b[k]) if b[k] < b[0] else None


def _packed_steps(forest, budgets, done, end, chunk=PACK_CHUNK):
    """Iterations [done, end) of a fresh forest on its current fused shape, in
    chunks; before each, the running trees go first, longest remaining budget
    first, so that a CTA's trees finish close together and no CTA keeps
    finished trees."""
    b = np.asarray(budgets, dtype=np.int64)
    while done < end:
        n = min(chunk, end - done)
        rem = b - done
        live = np.nonzero(rem > 0)[0]
        order = np.concatenate([live[np.argsort(-rem[live], kind="stable")], np.nonzero(rem <= 0)[0]])
        forest.dvc_forest_order(order.astype(np.int32), len(live))
        forest.dvc_mcts_step(n)
        done += n


def step_with_tail(forest, budgets, shape, sms, pack_per_sm=PACK_TREES_PER_SM, tail_per_sm=TAIL_TREES_PER_SM):
    """Search a fresh forest to the end of every budget: the given launch
    shape while many trees run; from at most pack_per_sm running trees per SM,
    the fused engine with several trees per CTA, repacked every PACK_CHUNK
    iterations; from at most tail_per_sm, one tree per CTA.  Results are those
    of any shape and order; re-tuning and repacking synchronise the device."""
    total = int(np.max(budgets))
    cut = tail_start(budgets, sms, pack_per_sm)
    if cut is None or cut >= total:
        forest.dvc_forest_tune(*shape)
        forest.dvc_mcts_step(total)
        return
    tail = tail_start(budgets, sms, tail_per_sm)
    tail = total if tail is None else max(cut, min(tail, total))
    if cut > 0:
        forest.dvc_forest_tune(*shape)
        forest.dvc_mcts_step(cut)
    if tail > cut:
        forest.dvc_forest_tune(*PACK_SHAPE)
        _packed_steps(forest, budgets, cut, tail)
    if total > tail:
        forest.dvc_forest_tune(*TAIL_SHAPE)
        _packed_steps(forest, budgets, tail, total)
    forest.dvc_forest_order(None)  # the next search starts from the default order again
