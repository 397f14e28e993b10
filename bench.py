#!/usr/bin/env python
"""Benchmark: Da Vinci Code MCTS decisions on GB300.

One step = one full decision batch of the 2-player/24-tile workload: 4,096
mid-game roots, each searched with 4,096 UCT iterations x 256 leaf playouts
(1,048,576 playouts per decision, 4.29e9 per step).  The step runs
dvc_forest_reset (re-plan and re-fill the determinization tables, reset the
trees), dvc_mcts_step (the CUDA-graph pipeline of determinization, select and
rollout kernels over overlapping chains) and dvc_root_stats (decisions).  The
timed steps keep no work counts; one more, untimed step of the same search
counts the random words and game steps.

Prints one JSON line.  `value` is playouts/s over all ranks (device-timed,
roots resident in HBM); `e2e` is the same metric through the public API with
host buffers: root states copied in from pinned memory and decisions copied
back inside each timed step.  `--impl reference` times the CPU oracle on a
bounded sample of the same workload on the host cores.

Launch: python bench.py [--gpus N --steps K --warmup W]; N > 1 under
torch.distributed.run (one rank per GPU, weak scaling: each rank searches its
own 4,096 trees).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# More hardware work queues than CUDA's default 8, before any CUDA call: the
# serving workload runs a dozen lane streams side by side, and the pipeline
# up to 24 chains.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

from paper_2403_10720_gb300.workloads import BATCHED, UNEVEN  # noqa: E402

# Algorithmic 32-bit integer operations by throughput class, per random word
# (Philox: 10 mul.lo/mul.hi, 10 xor + 5 key adds) and per game step of the
# two-player 24-tile playout apart from its words (the guess: hands, the
# unseen set and two population counts, the (slot, identity) split by one
# multiply-high and a reciprocal multiply, the slot's tile by a 12-bit
# select; the check, the reveal and the game-over test; the next seat's draw:
# pool, count, multiply-high, select, insert).
OPS_PER_WORD = {"alu": 15, "mul": 10, "popc": 0}
OPS_PER_STEP_2P24 = {"alu": 48, "mul": 5, "popc": 6}
# Per-SM, per-clock throughput of each class (CUDA C++ Programming Guide,
# arithmetic instruction throughput, compute capability 9.0 and 10.x): 64
# lanes for 32-bit integer add, logic, shift, compare and multiply, 16 for
# population count; an SM issues 4 warp instructions (128 lanes) per clock.
LANES_PER_CLOCK = {"alu": 64, "mul": 64, "popc": 16}
ISSUE_LANES_PER_CLOCK = 128
VALUE_MACS_PER_LEAF = 640 * 512 + 2 * 512 * 512 + 512 * 4  # dense layers of the value network
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
# DRAM bytes per launch of the pipeline's kernels at the default shape of the
# 4,096-tree workload (24 chains of 170 or 171 trees; 2 trees x 16 warps per
# rollout CTA), from ncu captures (cold cache) of the counting-free kernels,
# summarised under profiles/ with their commands.
PROFILED_SHAPE = (24, 2, 16)
DRAM_PER_LAUNCH = {"select": 346_507, "rollout": 74_384, "det": 200_512}
# Warp instructions per step of the same workload at that shape (4,096 trees
# x 4,096 iterations), summed over every kernel of the step by ncu
# (graph-level capture, instruction counts only), and lanes active per warp
# instruction; the capture is summarised under profiles/ with its command.
ISSUE_PROFILE = {"warp_instructions_per_step": 5.2416e11, "lanes_active_per_instruction": 23.73,
                 "source": "ncu smsp__inst_executed.sum / smsp__thread_inst_executed.sum over every kernel and "
                           "graph of one counting-free step at this shape (ncu summary under profiles/)"}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def shard_tree_ids(rank, n):
    """Weak scaling: rank r searches its own n trees, stream ids [r*n, (r+1)*n)."""
    return np.arange(rank * n, (rank + 1) * n, dtype=np.uint32)


def root_seed_of(rank, root_seed):
    """Each rank generates its own roots (no data exchange between ranks)."""
    return root_seed + 1000003 * rank


def max_over_ranks(seconds, dist, device):
    """The job's time for a phase is the slowest rank's (torch.distributed MAX)."""
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def value_net_roofline(dvc, ctx, peaks, peak_kind, leaves=65536, reps=5):
    """Time the value network (tensor cores) on `leaves` synthetic leaves."""
    import torch
    ctx.dvc_value_init(7)
    states = ctx.dvc_init_states(77, leaves)
    out = torch.empty((leaves, 4), dtype=torch.float32, device=states.device)
    ctx.dvc_value_eval(states, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        ctx.dvc_value_eval(states, out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    tflops = 2.0 * VALUE_MACS_PER_LEAF * leaves / (ms * 1e-3) / 1e12
    peak = float(peaks.get("bf16_tflops", 1900.0))
    return {"leaves": leaves, "ms": ms, "leaves_per_s": leaves / (ms * 1e-3),
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "peak_kind": f"bf16 burst ({peak_kind})"}}


def oracle_sample(w, n_trees, threads):
    """Search n_trees roots of the workload with the oracle, `threads` trees at a time."""
    import oracle
    cfg = oracle.OracleConfig(**w.config_kwargs())
    roots = oracle.init_states(cfg, w.root_seed, n_trees)
    budgets = w.budgets(n_trees)
    nxt = [0]
    lock = threading.Lock()

    def worker():
        while True:
            with lock:
                t = nxt[0]
                nxt[0] += 1
            if t >= n_trees:
                return
            oracle.mcts(cfg, roots[t], w.seed, t, int(budgets[t]))

    t0 = time.perf_counter()
    ths = [threading.Thread(target=worker) for _ in range(threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    dt = time.perf_counter() - t0
    playouts = int(budgets.sum()) * w.playouts
    return playouts, dt


def run_reference(args, w):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    n = cores  # one full tree per core per step: about 5 s of host work per step
    for _ in range(args.warmup):
        oracle_sample(w, min(n, 2), min(cores, 2))
    times, total = [], 0
    for _ in range(args.steps):
        p, dt = oracle_sample(w, n, cores)
        times.append(dt)
        total += p
    value = total / sum(times)
    p1, dt1 = oracle_sample(w, 1, 1)  # one tree on one thread
    sample = f"{n} of {w.n_trees} trees per step, each the full {w.budget} iterations x {w.playouts} playouts"
    line = {
        "impl": "reference", "metric": "playouts/s", "value": value, "unit": "playouts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "trees": w.n_trees, "iterations": w.budget, "playouts_per_leaf": w.playouts,
                   "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": "playouts/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "single_thread": {"value": p1 / dt1, "unit": "playouts/s", "decisions_per_s": 1.0 / dt1,
                                           "sample": "one tree on one host thread"}},
        "e2e": {"value": value, "unit": "playouts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "decisions_per_s": n * args.steps / sum(times),
    }
    print(json.dumps(line), flush=True)


def run_ours(args, w):
    import torch
    import torch.distributed as dist

    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build

    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    if world > 1:
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    if local == 0:
        build.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    ctx = dvc.Context(dvc.Config(**w.config_kwargs()), local)
    n = w.n_trees
    roots = ctx.dvc_init_states(root_seed_of(rank, w.root_seed), n)
    budgets = w.budgets()
    forest = dvc.Forest(ctx, roots, budgets, w.seed, tree_ids=shard_tree_ids(rank, n))
    # launch shape: the pipeline in CUDA graphs with the library's default
    # shape -- round(n / (1.12 SMs)) overlapping chains (at most 24), at least
    # 2 trees per rollout CTA, warps for one playout per thread -- unless overridden
    sms = props.multi_processor_count
    chains = args.chains or max(1, min(24, round(n / (1.12 * sms))))
    trees_per_cta = args.trees_per_cta or max(2, min(64, math.ceil(n / (chains * 0.85 * sms))))
    warps = args.warps or max(4, min(16, (trees_per_cta * w.playouts + 31) // 32))
    forest.dvc_forest_tune(2, trees_per_cta, warps, chains)
    if args.compact:
        receivers, donate_at = (int(x) for x in args.compact.split(","))
        forest.dvc_forest_compaction(receivers, donate_at)
    stats = torch.empty((n, 8), dtype=torch.int32, device=dev)
    work = torch.zeros(2, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    budget = int(budgets.max())
    playouts_per_step = int(budgets.sum()) * w.playouts

    def step(k0=None, k1=None):
        forest.dvc_forest_reset()
        if k0 is not None:
            k0.record(stream)
        forest.dvc_mcts_step(budget)
        if k1 is not None:
            k1.record(stream)
        forest.dvc_root_stats(out=stats)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.dvc_check()
    # the timed steps keep no work counts (instrumentation); the counts come
    # from one more, untimed step of the same (deterministic) search below
    forest.dvc_forest_count_work(False)
    step()

    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    ev = [(E(), E(), E(), E()) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    for k in range(args.steps):
        flush.fill_(k)  # L2 flush between timed steps (outside the step's events)
        s0, k0, k1, s1 = ev[k]
        s0.record(stream)
        step(k0, k1)
        s1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ctx.dvc_check()
    step_ms = [a.elapsed_time(b) for a, _, _, b in ev]
    kern_ms = [a.elapsed_time(b) for _, a, b, _ in ev]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        total_s = max_over_ranks(total_s, dist, dev)
    value = playouts_per_step * world * args.steps / total_s

    # end to end through the public API: host roots in, host decisions out
    host_roots = roots.cpu().pin_memory()
    host_stats = torch.empty((n, 8), dtype=torch.int32).pin_memory()
    dev_roots = torch.empty_like(roots)
    e2e_ms = []
    for k in range(max(1, args.steps)):
        flush.fill_(k)
        a, b = E(), E()
        a.record(stream)
        dev_roots.copy_(host_roots, non_blocking=True)
        forest.dvc_forest_reset(dev_roots)
        forest.dvc_mcts_step(budget)
        forest.dvc_root_stats(out=stats)
        host_stats.copy_(stats, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_s = sum(e2e_ms) / 1e3
    if world > 1:
        e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_value = playouts_per_step * world * len(e2e_ms) / e2e_s
    ctx.dvc_check()
    decisions = host_stats.numpy()
    # work of one step: the same search with the counters kept
    forest.dvc_forest_count_work(True)
    forest.dvc_forest_work(out=work)
    step()
    forest.dvc_forest_work(out=work)
    torch.cuda.synchronize()
    ctx.dvc_check()
    words_per_step = int(work[0].item())
    game_steps_per_step = int(work[1].item())

    traffic = None
    if (chains, trees_per_cta, warps) == PROFILED_SHAPE and n == 4096 and not args.compact:
        traffic = (budget * chains * (DRAM_PER_LAUNCH["select"] + DRAM_PER_LAUNCH["rollout"])
                   + -(-budget // 64) * chains * DRAM_PER_LAUNCH["det"])
    peaks, peak_kind = _measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    kern_mean_s = sum(kern_ms) / len(kern_ms) / 1e3
    # ALU roofline in game steps: the algorithmic integer operations of one
    # step (its own plus its share of random words), by class; the bound is
    # the class that needs the most clocks per SM at its documented rate
    wps = words_per_step / max(game_steps_per_step, 1.0)
    ops = {c: OPS_PER_STEP_2P24[c] + wps * OPS_PER_WORD[c] for c in LANES_PER_CLOCK}
    clocks_per_step = {c: ops[c] / LANES_PER_CLOCK[c] for c in ops}
    clocks_per_step["issue"] = sum(ops.values()) / ISSUE_LANES_PER_CLOCK
    bound_class = max(clocks_per_step, key=clocks_per_step.get)
    peak_gsteps = props.multi_processor_count * sm_max * 1e6 / clocks_per_step[bound_class] / 1e9
    achieved_gsteps = game_steps_per_step / kern_mean_s / 1e9
    issue = None
    if (chains, trees_per_cta, warps) == PROFILED_SHAPE and n == 4096 and budget == 4096 and not args.compact:
        issue = {"utilisation": ISSUE_PROFILE["warp_instructions_per_step"] / (
                     props.multi_processor_count * 4 * sm_max * 1e6 * (sum(step_ms) / len(step_ms) / 1e3)),
                 "lanes_active_per_instruction": ISSUE_PROFILE["lanes_active_per_instruction"],
                 "warp_instructions_per_playout": ISSUE_PROFILE["warp_instructions_per_step"] / playouts_per_step,
                 "source": ISSUE_PROFILE["source"]} if ISSUE_PROFILE else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": "playouts/s", "value": value, "unit": "playouts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "trees": n, "iterations": w.budget, "playouts_per_leaf": w.playouts,
                   "players": w.nplayers, "tiles": w.ntiles, "d_max": w.d_max,
                   "engine": f"pipeline, {trees_per_cta} trees x {warps} warps per rollout CTA, {chains} chains, "
                             "CUDA graph" + (f", lane compaction {args.compact}" if args.compact else ""),
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
        "decisions_per_s": n * world * args.steps / total_s,
        "kernel_ms": sum(kern_ms) / len(kern_ms),
        "words_per_playout": words_per_step / playouts_per_step,
        "game_steps_per_playout": game_steps_per_step / playouts_per_step,
        "game_steps_per_s": game_steps_per_step * world * args.steps / total_s,
        "issue_slots": issue,
        "e2e": {"value": e2e_value, "unit": "playouts/s", "h2d_bytes_per_step": int(host_roots.numel()),
                "d2h_bytes_per_step": int(host_stats.numel() * 4)},
        # kernels per step: forest reset, pipeline begin, per 64-iteration chunk one
        # determinization launch per chain, per iteration (select + rollout) x chains,
        # final backprop, root stats
        "gpu_launches": args.steps * (4 + chains * (-(-budget // 64)) + 2 * budget * chains),
        "roofline": {"bound": "alu", "achieved": achieved_gsteps, "peak": peak_gsteps, "unit": "Gstep/s",
                     "frac": achieved_gsteps / peak_gsteps, "traffic": traffic,
                     "peak_kind": f"{props.multi_processor_count} SMs x {sm_max:.0f} MHz ({peak_kind} clock) / "
                                  f"{clocks_per_step[bound_class]:.3f} SM clocks per game step ({bound_class} "
                                  "class bound)",
                     "ops_per_step": {c: round(v, 2) for c, v in ops.items()},
                     "clocks_per_step": {c: round(v, 4) for c, v in clocks_per_step.items()},
                     "work": "game steps (a playout guess with its resolution, continue coin and the next seat's "
                             "draw), counted by the playout kernels; per step the algorithmic integer operations "
                             "by class, Philox words included",
                     "launch": "one dvc_mcts_step: the CUDA-graph pipeline (determinize-ahead, select, rollout "
                               "kernels of all chains)",
                     "traffic_source": "ncu dram__bytes per kernel launch (cold cache) x launches per step; null "
                                       "when the launch shape differs from the profiled one"},
        "clocks": clk,
        "first_decision": int(decisions[0][0]),
    }
    if rank == 0:
        line["value_net"] = value_net_roofline(dvc, ctx, peaks, peak_kind)
    if rank == 0 and world == 1 and not args.no_extras:
        # the other configurations, each bounded in time: one step of the
        # uneven forest, a serving run, the value network against playouts
        forest.close()
        del flush
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        for key, fn in (("uneven", lambda: measure_uneven(UNEVEN, steps=1, warmup=1)),
                        ("serve", lambda: serve_games(10_000, 400.0, 10.0, 64.0, 100_000, 256)),
                        ("value_vs_rollout", value_vs_rollout)):
            try:
                line[key] = fn()
            except Exception as exc:  # the main measurement above stands; record what failed
                line[key] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.empty_cache()
        line["extras_wall_s"] = time.perf_counter() - t0
    if world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        p, dt = oracle_sample(w, cores, cores)
        line["cpu_baseline"] = {"value": p / dt, "unit": "playouts/s", "cores": cores, "kind": "oracle",
                                "sample": f"{cores} of {w.n_trees} trees, full {w.budget} iterations x "
                                          f"{w.playouts} playouts each, one tree per host thread"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_uneven(w, steps=1, warmup=1, trees=0, iterations=0, shape=None, warmup_cap=64):
    """The uneven forest (16,384 four-player joker trees, budgets 1k-100k):
    every tree searches its whole budget; one
    step = all trees.  The launch shape comes from the autotuner unless given;
    the tail of long budgets runs on the fused engine (autotune.step_with_tail).
    Warm-up steps run with budgets capped at warmup_cap iterations (graph
    capture, kernel attributes).  Returns a dict of the measurement."""
    import torch

    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import autotune, build
    build.build()
    ctx = dvc.Context(dvc.Config(**w.config_kwargs()), 0)
    n = trees or w.n_trees
    roots = ctx.dvc_init_states(w.root_seed, n)
    budgets = w.budgets(n)
    if iterations:  # small profiling cases: budgets capped
        budgets = np.minimum(budgets, iterations).astype(np.int32)
    if shape is None:
        shape = autotune.tune(dvc, ctx, roots, budgets, w.seed, scale=0.02)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cut = autotune.tail_start(budgets, sms, autotune.PACK_TREES_PER_SM)
    cut_tail = autotune.tail_start(budgets, sms)
    if warmup:
        capped = np.minimum(budgets, warmup_cap).astype(np.int32)
        f0 = dvc.Forest(ctx, roots, capped, w.seed)
        f0.dvc_forest_tune(*shape)
        for _ in range(warmup):
            f0.dvc_forest_reset()
            autotune.step_with_tail(f0, capped, shape, sms)
        torch.cuda.synchronize()
        f0.close()
    forest = dvc.Forest(ctx, roots, budgets, w.seed)
    forest.dvc_forest_tune(*shape)
    stats = torch.empty((n, 8), dtype=torch.int32, device=roots.device)
    work = torch.zeros(2, dtype=torch.int64, device=roots.device)
    forest.dvc_forest_work(out=work)
    ev = []
    clocks = ClockSampler(0)
    clocks.start()
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        forest.dvc_forest_reset()
        # the tuned shape while many trees run, then packed fused CTAs, then one tree per CTA
        autotune.step_with_tail(forest, budgets, shape, sms)
        forest.dvc_root_stats(out=stats)
        b.record()
        ev.append((a, b))
    torch.cuda.synchronize()
    clk = clocks.stop()
    forest.dvc_forest_work(out=work)
    ctx.dvc_check()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(ms) / 1e3
    playouts = int(budgets.sum()) * w.playouts * steps
    st = stats.cpu().numpy()
    assert (st[:, 6] == budgets).all()
    forest.close()
    ctx.close()
    return {"workload": w.name if n == w.n_trees and not iterations else f"{w.name}_first{n}_cap{iterations}",
            "playouts_per_s": playouts / total_s, "decisions_per_s": n * steps / total_s,
            "ms_per_step": 1e3 * total_s / steps, "steps": steps,
            "game_steps_per_s": int(work[1].item()) / total_s,
            "words_per_playout": int(work[0].item()) / playouts, "trees": n,
            "iterations_total": int(budgets.sum()), "budget_range": [int(budgets.min()), int(budgets.max())],
            "playouts_per_leaf": w.playouts, "players": w.nplayers, "tiles": w.ntiles,
            "launch_shape": list(shape),
            "tail": {"from_iteration": cut, "launch_shape": list(autotune.PACK_SHAPE),
                     "repacked_every": autotune.PACK_CHUNK,
                     "then": {"from_iteration": cut_tail, "launch_shape": list(autotune.TAIL_SHAPE)}},
            "clocks": clk}


def run_uneven(args, w):
    """The uneven forest on its own (one JSON line)."""
    m = measure_uneven(w, steps=args.steps, warmup=args.warmup, trees=args.trees, iterations=args.iterations,
                       shape=(args.engine or 2, args.trees_per_cta, args.warps, args.chains)
                       if (args.engine or args.chains or args.trees_per_cta or args.warps) else None)
    print(json.dumps({
        "metric": "playouts/s", "value": m["playouts_per_s"], "unit": "playouts/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {k: m[k] for k in ("workload", "trees", "iterations_total", "budget_range", "playouts_per_leaf",
                                     "players", "tiles", "launch_shape", "tail")} |
                  {"l2": "working set (node arenas) far above L2"},
        "decisions_per_s": m["decisions_per_s"], "game_steps_per_s": m["game_steps_per_s"], "clocks": m["clocks"]}),
          flush=True)


def _crossing(xs, ys, level=0.5):
    """x where the piecewise-linear curve through (xs, ys) first reaches
    `level` (xs ascending), or None if it does not within the range."""
    for (x0, y0), (x1, y1) in zip(zip(xs, ys), zip(xs[1:], ys[1:])):
        if (y0 - level) * (y1 - level) <= 0 and y1 != y0:
            return x0 + (level - y0) * (x1 - x0) / (y1 - y0)
        if y0 == level:
            return x0
    return None


def value_vs_rollout(train_states=10_000_000, epochs=4, games=2000, rollout_budget=256,
                     value_budgets=(128, 192, 256, 384), hbm_gb=4.0):
    """Value network against playouts: the network trained on the GPU (states of the 2-player
    24-tile root generator labelled by 1,024 playouts each), its held-out
    win-probability error against rollout estimates, then games of the value
    agent at several iteration budgets against the playout agent (32 playouts
    per leaf) at rollout_budget, with 95% intervals; the GPU time per decision
    of each agent; and the budget, in iterations and in GPU time relative to
    the playout agent, at which the value agent wins half the games."""
    import torch

    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build, selfplay
    from paper_2403_10720_gb300 import value_train as vt
    build.build()
    w = BATCHED
    kw = dict(w.config_kwargs(), playouts=32)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    ctx.dvc_value_init(1)
    t0 = time.perf_counter()
    states, labels = vt.make_dataset(ctx, train_states, root_seed=1001)
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t0
    t0 = time.perf_counter()
    curve = vt.train(ctx, states, labels, epochs=epochs, batch=8192, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del states, labels
    hs, hl = vt.make_dataset(ctx, 16384, root_seed=2002)
    err = {"net": vt.mean_abs_error(ctx.dvc_value_eval(hs), hl, hs)}
    for k in (16, 64, 256):
        err[f"playouts_{k}"] = vt.mean_abs_error(vt.rollout_estimate(ctx, hs, k), hl, hs)
    roots = ctx.dvc_init_states(w.root_seed, 4096)
    agree = selfplay.move_agreement(ctx, dvc, roots, rollout_budget, 16 * rollout_budget, seed=7)
    half = {k: 1.96 * math.sqrt(max(v * (1 - v), 1e-12) / agree["positions"]) for k, v in agree.items()
            if k.endswith("strong") or k == "value_vs_rollout"}
    agree["ci95_half_width"] = half

    def us_per_decision(budget, mode):
        f = dvc.Forest(ctx, roots, [budget] * 4096, 5)
        f.dvc_mcts_step(budget, mode=mode)
        f.dvc_forest_reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        f.dvc_mcts_step(budget, mode=mode)
        b.record()
        torch.cuda.synchronize()
        f.close()
        return a.elapsed_time(b) * 1e3 / 4096
    t_roll = us_per_decision(rollout_budget, dvc.DVC_MODE_ROLLOUT)
    t_val = {b: us_per_decision(b, dvc.DVC_MODE_VALUE) for b in value_budgets}
    gctx = dvc.Context(dvc.Config(**dict(kw, max_predraw=0)), 0)
    gctx.dvc_value_init(1)
    gctx.dvc_value_params(ctx.dvc_value_params())
    server = dvc.Server(gctx, int(hbm_gb * (1 << 30)), max(max(value_budgets), rollout_budget), value_share_pct=50,
                        seed=9)
    points = []
    t0 = time.perf_counter()
    for b in value_budgets:
        g = selfplay.play_games(gctx, server, games, rollout_budget, root_seed=3003, seed=11, value_budget=b,
                                poll_iters=max(b, rollout_budget))
        points.append({"value_iterations": b, "win_rate": g["value_win_rate"], "ci95": g["ci95"],
                       "games_finished": g["games_finished"], "value_us_per_decision": t_val[b]})
    t_games = time.perf_counter() - t0
    server.close()
    gctx.dvc_check()
    ctx.dvc_check()
    xs = [p["value_iterations"] for p in points]
    mid = _crossing(xs, [p["win_rate"] for p in points])
    lo = _crossing(xs, [p["ci95"][1] for p in points])   # upper edge reaches 0.5 first
    hi = _crossing(xs, [p["ci95"][0] for p in points])
    t_at = (lambda x: None if x is None else float(np.interp(x, xs, [t_val[b] for b in xs])))
    return {
        "workload": "2p24_value_vs_playouts_selfplay", "games_per_point": games, "players": 2, "tiles": 24,
        "rollout_iterations": rollout_budget, "playouts_per_leaf": 32, "points": points,
        "rollout_us_per_decision": t_roll,
        "value_iterations_at_50pct": mid, "value_iterations_at_50pct_ci95": [lo, hi],
        "gpu_time_ratio_at_50pct": None if mid is None else t_at(mid) / t_roll,
        "gpu_time_ratio_at_50pct_ci95": [None if x is None else t_at(x) / t_roll for x in (lo, hi)],
        "winprob_abs_err_heldout": err, "move_agreement": agree,
        "train": {"states": train_states, "label_playouts": 1024, "epochs": epochs, "label_s": t_label,
                  "train_s": t_train, "loss_first_epoch": curve[0], "loss_last_epoch": curve[-1]},
        "games_wall_s": t_games,
    }


def run_selfplay(args):
    """The value network against playouts: train it on states labelled by
    1,024-playout estimates, measure its win-probability error and move
    agreement, then play games between the value agent and the playout agent
    at equal iteration budgets (one line of JSON)."""
    import numpy as np
    import torch

    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build, selfplay
    from paper_2403_10720_gb300 import value_train as vt
    build.build()
    w = BATCHED
    kw = dict(w.config_kwargs(), playouts=32)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    ctx.dvc_value_init(1)
    t0 = time.perf_counter()
    states, labels = vt.make_dataset(ctx, args.train_states, root_seed=1001)
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t0
    t0 = time.perf_counter()
    curve = vt.train(ctx, states, labels, epochs=args.epochs, batch=8192, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del states, labels
    hs, hl = vt.make_dataset(ctx, 16384, root_seed=2002)
    err = {"net": vt.mean_abs_error(ctx.dvc_value_eval(hs), hl, hs)}
    for k in (16, 64, 256):
        err[f"playouts_{k}"] = vt.mean_abs_error(vt.rollout_estimate(ctx, hs, k), hl, hs)
    roots = ctx.dvc_init_states(w.root_seed, 4096)
    agree = selfplay.move_agreement(ctx, dvc, roots, args.move_budget, 16 * args.move_budget, seed=7)
    # GPU time per decision of each agent on the same 4,096 positions
    per_dec = {}
    for name, mode in (("value", dvc.DVC_MODE_VALUE), ("rollout", dvc.DVC_MODE_ROLLOUT)):
        f = dvc.Forest(ctx, roots, [args.move_budget] * 4096, 5)
        f.dvc_mcts_step(args.move_budget, mode=mode)
        f.dvc_forest_reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        f.dvc_mcts_step(args.move_budget, mode=mode)
        b.record()
        torch.cuda.synchronize()
        per_dec[name] = a.elapsed_time(b) / 4096
        f.close()
    # games: fresh deals of the same variant
    gctx = dvc.Context(dvc.Config(**dict(kw, max_predraw=0)), 0)
    params = ctx.dvc_value_params()
    gctx.dvc_value_init(1)
    gctx.dvc_value_params(params)
    server = dvc.Server(gctx, int(args.hbm_gb * (1 << 30)), args.move_budget, value_share_pct=50, seed=9)
    games = selfplay.play_games(gctx, server, args.games, args.move_budget, root_seed=3003, seed=11,
                                poll_iters=args.move_budget)
    # the value agent with half the iterations against the full-budget playout agent
    half = selfplay.play_games(gctx, server, args.games, args.move_budget, root_seed=3003, seed=11,
                               value_budget=args.move_budget // 2, poll_iters=args.move_budget)
    server.close()
    print(json.dumps({
        "metric": "value-agent win rate", "value": games["value_win_rate"], "unit": "fraction of games",
        "n_gpus": 1, "higher_is_better": True, "dtype": "bf16 net / u32 playouts", "data": "synthetic",
        "config": {"workload": "2p24_value_vs_playouts_selfplay", "train_states": args.train_states,
                   "label_playouts": 1024, "epochs": args.epochs, "games": args.games,
                   "iterations_per_move": args.move_budget, "playouts_per_leaf": 32, "players": 2, "tiles": 24},
        "ci95": games["ci95"], "fair_share": games["fair_share"], "games_finished": games["games_finished"],
        "turns": games["turns"], "selfplay_decisions_per_s": games["decisions_per_s"],
        "selfplay_wall_s": games["wall_s"],
        "value_half_budget": {"value_iterations": args.move_budget // 2, "rollout_iterations": args.move_budget,
                              "value_win_rate": half["value_win_rate"], "ci95": half["ci95"]},
        "winprob_abs_err_heldout": err, "move_agreement": agree,
        "gpu_ms_per_decision": per_dec,
        "train": {"label_s": t_label, "train_s": t_train, "loss_first_epoch": curve[0], "loss_last_epoch": curve[-1]},
    }), flush=True)


def run_policy(args):
    """The ordering-aware playout policy against the uniform one: games
    between the two playout agents at equal iteration budgets, and the search
    throughput of each policy on the batched workload (one line of JSON)."""
    import dataclasses

    import torch

    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build, selfplay
    build.build()
    w = BATCHED
    speed = {}
    for policy in (0, 1):
        ctx = dvc.Context(dvc.Config(**dict(w.config_kwargs(), policy=policy)), 0)
        n, it = w.n_trees, 512
        roots = ctx.dvc_init_states(w.root_seed, n)
        f = dvc.Forest(ctx, roots, [it] * n, w.seed)
        f.dvc_mcts_step(it)
        f.dvc_forest_reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        f.dvc_mcts_step(it)
        b.record()
        torch.cuda.synchronize()
        ctx.dvc_check()
        ms = a.elapsed_time(b)
        speed["ordered" if policy else "uniform"] = {"playouts_per_s": n * it * w.playouts / (ms * 1e-3),
                                                     "ms": ms, "trees": n, "iterations": it}
        f.close()
    kw = dict(w.config_kwargs(), playouts=32, max_predraw=0)
    ctx_u = dvc.Context(dvc.Config(**dict(kw, policy=0)), 0)
    ctx_o = dvc.Context(dvc.Config(**dict(kw, policy=1)), 0)
    hbm = int(args.hbm_gb * (1 << 30)) // 2
    srv_u = dvc.Server(ctx_u, hbm, args.move_budget, seed=9)
    srv_o = dvc.Server(ctx_o, hbm, args.move_budget, seed=9)
    games = selfplay.play_agents(ctx_u, (srv_o, dvc.DVC_MODE_ROLLOUT, args.move_budget),
                                 (srv_u, dvc.DVC_MODE_ROLLOUT, args.move_budget), args.games, root_seed=3003, seed=11,
                                 poll_iters=args.move_budget)
    srv_u.close()
    srv_o.close()
    print(json.dumps({
        "metric": "ordered-policy agent win rate", "value": games["a_win_rate"], "unit": "fraction of games",
        "n_gpus": 1, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "2p24_ordered_vs_uniform_playouts_selfplay", "games": args.games,
                   "iterations_per_move": args.move_budget, "playouts_per_leaf": 32, "players": 2, "tiles": 24},
        "ci95": games["ci95"], "fair_share": games["fair_share"], "games_finished": games["games_finished"],
        "turns": games["turns"], "selfplay_decisions_per_s": games["decisions_per_s"],
        "search_throughput": speed,
    }), flush=True)


def run_fulltree(args):
    """The full game tree of Fig. 2a (a correct guess keeps the turn; STOP is
    an action) against the paper's simplified tree, as two agents playing the
    full game at equal iteration budgets (one line of JSON)."""
    import torch

    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build, selfplay
    build.build()
    w = BATCHED
    kw = dict(w.config_kwargs(), playouts=32, max_predraw=0)
    game = dvc.Context(dvc.Config(**dict(kw, tree_continue=1)), 0)
    ctx_full = dvc.Context(dvc.Config(**dict(kw, tree_continue=1)), 0)
    ctx_simple = dvc.Context(dvc.Config(**dict(kw, tree_continue=0)), 0)
    hbm = int(args.hbm_gb * (1 << 30)) // 2
    srv_full = dvc.Server(ctx_full, hbm, args.move_budget, seed=9)
    srv_simple = dvc.Server(ctx_simple, hbm, args.move_budget, seed=9)
    games = selfplay.play_agents(game, (srv_full, dvc.DVC_MODE_ROLLOUT, args.move_budget),
                                 (srv_simple, dvc.DVC_MODE_ROLLOUT, args.move_budget), args.games, root_seed=3003,
                                 seed=11, poll_iters=args.move_budget)
    srv_full.close()
    srv_simple.close()
    # search throughput of each tree on the batched roots
    speed = {}
    for name, cont in (("full", 1), ("simplified", 0)):
        ctx = dvc.Context(dvc.Config(**dict(w.config_kwargs(), tree_continue=cont)), 0)
        roots = ctx.dvc_init_states(w.root_seed, w.n_trees)
        f = dvc.Forest(ctx, roots, [512] * w.n_trees, w.seed)
        f.dvc_mcts_step(512)
        f.dvc_forest_reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        f.dvc_mcts_step(512)
        b.record()
        torch.cuda.synchronize()
        ctx.dvc_check()
        speed[name] = {"playouts_per_s": w.n_trees * 512 * w.playouts / (a.elapsed_time(b) * 1e-3)}
        f.close()
    print(json.dumps({
        "metric": "full-tree agent win rate", "value": games["a_win_rate"], "unit": "fraction of games",
        "n_gpus": 1, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "2p24_full_vs_simplified_tree_selfplay", "games": args.games,
                   "iterations_per_move": args.move_budget, "playouts_per_leaf": 32, "players": 2, "tiles": 24,
                   "game": "full (a correct guess keeps the turn)"},
        "ci95": games["ci95"], "fair_share": games["fair_share"], "games_finished": games["games_finished"],
        "moves": games["turns"], "decisions": {"full": games["decisions_a"], "simplified": games["decisions_b"]},
        "selfplay_decisions_per_s": games["decisions_per_s"], "search_throughput": speed,
    }), flush=True)


def run_vanilla(args):
    """Vanilla MCTS-dvc (the root's children are plausible-number sets, Sec.
    III-A) against the paper's MCTS-dvc on two-player 24-tile positions: how
    the root's statistics spread over sets, search throughput, agreement with
    a strong MCTS-dvc search (16x the iterations), and games between the two
    agents at equal iteration budgets (one line of JSON)."""
    import numpy as np
    import torch

    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build, selfplay
    build.build()
    w = BATCHED
    B = args.move_budget
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    positions = {}
    for pos, mp in (("opening", 0), ("mid_game", w.config_kwargs()["max_predraw"])):
        kw = dict(w.config_kwargs(), max_predraw=mp)
        res = {}
        ctx0 = dvc.Context(dvc.Config(**kw), 0)
        roots = ctx0.dvc_init_states(w.root_seed, w.n_trees)
        strong = dvc.Forest(ctx0, roots, [16 * B] * w.n_trees, w.seed + 1)
        strong.dvc_mcts_step(16 * B)
        ref = strong.dvc_root_stats()[:, 0].cpu().numpy()
        strong.close()
        for name, van in (("vanilla", 1), ("mcts_dvc", 0)):
            ctx = dvc.Context(dvc.Config(**dict(kw, vanilla=van)), 0)
            f = dvc.Forest(ctx, roots, [B] * w.n_trees, w.seed)
            f.dvc_mcts_step(B)
            f.dvc_forest_reset()
            torch.cuda.synchronize()
            a, b = E(), E()
            a.record()
            f.dvc_mcts_step(B)
            b.record()
            torch.cuda.synchronize()
            st = f.dvc_root_stats().cpu().numpy().astype(np.int64)
            ctx.dvc_check()
            f.close()
            res[name] = {
                "playouts_per_s": w.n_trees * B * w.playouts / (a.elapsed_time(b) * 1e-3),
                "root_children_mean": float(st[:, 4].mean()),
                "root_children_max": int(st[:, 4].max()),
                "visits_per_root_child": float((st[:, 3] / np.maximum(st[:, 4], 1)).mean()),
                "best_action_visit_share": float((st[:, 1] / np.maximum(st[:, 3], 1)).mean()),
                "agreement_with_strong_mcts_dvc": float((st[:, 0] == ref).mean()),
            }
        positions[pos] = res
    kw = dict(w.config_kwargs(), playouts=32, max_predraw=0)
    game = dvc.Context(dvc.Config(**kw), 0)
    van = dvc.Context(dvc.Config(**dict(kw, vanilla=1)), 0)
    games = selfplay.play_forest_agents(game, (van, B), (game, B), args.games, root_seed=3003, seed=11)
    print(json.dumps({
        "metric": "vanilla agent win rate", "value": games["a_win_rate"], "unit": "fraction of games",
        "n_gpus": 1, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "2p24_vanilla_vs_mcts_dvc", "games": args.games, "iterations_per_move": B,
                   "playouts_per_leaf_games": 32, "trees_per_position_kind": w.n_trees,
                   "playouts_per_leaf_search": w.playouts, "strong_iterations": 16 * B, "players": 2, "tiles": 24},
        "ci95": games["ci95"], "fair_share": games["fair_share"], "games_finished": games["games_finished"],
        "moves": games["turns"], "decisions": {"vanilla": games["decisions_a"], "mcts_dvc": games["decisions_b"]},
        "selfplay_decisions_per_s": games["decisions_per_s"], "positions": positions,
    }), flush=True)


def run_scaling(args):
    """The paper's scaling sweeps (Sec. IV: simulations per second against
    CPU threads, GPU threads and warps; weak scaling) repeated for this
    implementation on the 2-player 24-tile batched workload (one JSON line)."""
    import dataclasses

    import numpy as np
    import torch

    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build
    build.build()
    w = BATCHED
    ctx = dvc.Context(dvc.Config(**w.config_kwargs()), 0)
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = E(), E()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps / 1e3

    # GPU threads: standalone leaf-parallel playouts, 256 per leaf, one thread per playout
    leaves_all = ctx.dvc_init_states(w.root_seed, 65536)
    ids = torch.arange(65536, dtype=torch.int32, device=leaves_all.device)
    threads = []
    for n in (1, 4, 16, 64, 256, 1024, 4096, 16384, 65536):
        sec = timed(lambda: ctx.dvc_rollout_batch(leaves_all[:n], 256, 5, ids[:n], ids[:n]))
        threads.append({"leaves": n, "playouts": n * 256, "seconds": sec, "playouts_per_s": n * 256 / sec})
    # warps per rollout CTA: the pipeline at 16 chains x 2 trees, 4,096 trees x 256 iterations
    roots = ctx.dvc_init_states(w.root_seed, w.n_trees)
    warps = []
    for W in (1, 2, 4, 8, 16, 32):
        f = dvc.Forest(ctx, roots, [256] * w.n_trees, w.seed)
        f.dvc_forest_tune(2, 2, W, 16)

        def step():
            f.dvc_forest_reset()
            f.dvc_mcts_step(256)
        sec = timed(step, reps=2)
        warps.append({"warps_per_cta": W, "seconds": sec, "playouts_per_s": w.n_trees * 256 * w.playouts / sec})
        f.close()
    # weak scaling: fixed work per tree (256 iterations x 256 playouts), growing forest
    weak = []
    for n in (38, 76, 152, 304, 608, 1216, 2432, 4096, 8192):
        r = ctx.dvc_init_states(w.root_seed, n)
        f = dvc.Forest(ctx, r, [256] * n, w.seed)

        def step():
            f.dvc_forest_reset()
            f.dvc_mcts_step(256)
        sec = timed(step, reps=2)
        weak.append({"trees": n, "seconds": sec, "playouts_per_s": n * 256 * w.playouts / sec})
        f.close()
    ctx.dvc_check()
    # CPU threads: the oracle, one 256-iteration tree per thread
    small = dataclasses.replace(w, budget=256)
    cpu = []
    cores = os.cpu_count() or 1
    for t in sorted({1, 2, 4, 8, 16, cores}):
        if t > cores:
            continue
        p, dt = oracle_sample(small, t, t)
        cpu.append({"threads": t, "playouts_per_s": p / dt})
    print(json.dumps({"metric": "scaling sweeps", "workload": w.name, "gpu_threads": threads,
                      "gpu_warps_per_rollout_cta": warps, "gpu_weak_scaling": weak, "cpu_oracle_threads": cpu}),
          flush=True)


SERVE_VARIANTS = [  # the serving workload: 2-4 players, 24- and 26-tile games (26 tiles: with the two jokers)
    dict(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5),
    dict(nplayers=3, ntiles=24, deal=4, max_predraw=6, max_revealed=3),
    dict(nplayers=4, ntiles=24, deal=3, max_predraw=6, max_revealed=3),
    dict(nplayers=2, ntiles=26, deal=4, max_predraw=10, max_revealed=5),
    dict(nplayers=3, ntiles=26, deal=4, max_predraw=6, max_revealed=3),
    dict(nplayers=4, ntiles=26, deal=3, max_predraw=8, max_revealed=3),
]


def serve_games(games, rate, window_s, hbm_gb, max_budget, poll_iters, value_frac=0.5, value_share_pct=35):
    """Serving: one server over six game variants sharing an HBM
    budget, Poisson arrivals of move queries from `games` concurrent games,
    value and rollout modes mixed per query.  Returns the driver's dict plus
    the server's slot layout."""
    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build, serving
    build.build()
    ctxs = []
    for i, kw in enumerate(SERVE_VARIANTS):
        c = dvc.Context(dvc.Config(**dict(kw, playouts=32)), 0)
        c.dvc_value_init(100 + i)
        ctxs.append(c)
    server = dvc.Server(ctxs, int(hbm_gb * (1 << 30)), max_budget, value_share_pct=value_share_pct, seed=5)
    lanes = server.dvc_server_lanes()
    out = serving.game_serving_run(server, ctxs, games, rate, window_s, budget_lo=1000, budget_hi=max_budget,
                                   value_frac=value_frac, seed=6, iterations_per_poll=poll_iters)
    for c in ctxs:
        c.dvc_check()
    after = server.dvc_server_lanes()
    server.close()
    out["lanes"] = [{"variant": f"{l['players']}p{l['tiles']}", "mode": ("rollout", "value")[l["mode"]],
                     "slots": l["slots"], "steps": a["steps"],
                     "us_per_iteration": a["step_us"] / poll_iters if a["steps"] else None}
                    for l, a in zip(lanes, after)]
    out["hbm_gb"] = hbm_gb
    out["iterations_per_poll"] = poll_iters
    out["budget_range"] = [1000, max_budget]
    out["value_frac"] = value_frac
    out["playouts_per_leaf"] = 32
    return out


def run_serve(args):
    """The serving workload on its own: Poisson arrivals of move queries from concurrent
    games of six variants into one device-resident server (one JSON line)."""
    out = serve_games(args.games_live, args.rate, args.window, args.hbm_gb, args.max_budget, args.poll_iters)
    print(json.dumps({
        "metric": "decisions/s", "value": out["decisions_per_s"], "unit": "decisions/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "u32 playouts / bf16 net", "data": "synthetic",
        "config": {"workload": "serving_6variants_poisson", "games": out["games"], "rate_per_s": args.rate,
                   "arrival_window_s": args.window, "budget_range": out["budget_range"],
                   "value_frac": out["value_frac"], "playouts_per_leaf": 32, "hbm_gb": args.hbm_gb,
                   "iterations_per_poll": args.poll_iters},
        **{k: out[k] for k in ("queries", "wall_s", "moves_played", "games_redealt", "p50_ms", "p99_ms", "by_mode",
                               "by_variant", "lanes", "polls", "host_s")}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the uneven-forest, serving and value-vs-playout sub-measurements")
    ap.add_argument("--trees", type=int, default=0, help="override the tree count (small profiling cases)")
    ap.add_argument("--iterations", type=int, default=0, help="override the iterations per tree")
    ap.add_argument("--chains", type=int, default=0, help="pipeline chains (launch shape only; 0 = default)")
    ap.add_argument("--trees-per-cta", type=int, default=0, help="pipeline trees per rollout CTA (0 = default)")
    ap.add_argument("--warps", type=int, default=0, help="warps per rollout CTA (0 = default)")
    ap.add_argument("--compact", default="", help="lane compaction 'receivers,donate_at' (default off)")
    ap.add_argument("--engine", type=int, default=0, help="uneven: 1 fused, 2 pipeline (launch shape only)")
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "uneven", "serve", "selfplay", "policy", "scaling", "fulltree", "vanilla"])
    ap.add_argument("--train-states", type=int, default=10_000_000, help="selfplay: training states")
    ap.add_argument("--epochs", type=int, default=4, help="selfplay: training epochs")
    ap.add_argument("--games", type=int, default=10_000, help="selfplay: games between the two agents")
    ap.add_argument("--move-budget", type=int, default=256, help="selfplay: UCT iterations per move")
    ap.add_argument("--games-live", type=int, default=10_000, help="serve: concurrent games")
    ap.add_argument("--window", type=float, default=10.0, help="serve: seconds of query arrivals")
    ap.add_argument("--rate", type=float, default=400.0, help="serve: Poisson arrival rate (queries/s)")
    ap.add_argument("--max-budget", type=int, default=100000, help="serve: largest query budget")
    ap.add_argument("--hbm-gb", type=float, default=64.0, help="serve: HBM budget for resident searches")
    ap.add_argument("--poll-iters", type=int, default=256, help="serve: iterations per poll")
    args = ap.parse_args()
    if args.workload == "uneven":
        run_uneven(args, UNEVEN)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "scaling":
        run_scaling(args)
        return
    if args.workload in ("selfplay", "policy", "fulltree", "vanilla"):
        if args.hbm_gb == 64.0:
            args.hbm_gb = 4.0
        {"selfplay": run_selfplay, "policy": run_policy, "fulltree": run_fulltree,
         "vanilla": run_vanilla}[args.workload](args)
        return
    w = BATCHED
    if args.trees or args.iterations:
        import dataclasses
        n, it = args.trees or w.n_trees, args.iterations or w.budget
        w = dataclasses.replace(w, n_trees=n, budget=it, name=f"2p24_{n}trees_{it}it_{w.playouts}po")
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
