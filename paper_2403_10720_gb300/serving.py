"""Drive a dvc_server with Poisson arrivals of move queries and measure
latency (submission to result) and decisions per second."""
import time

import numpy as np


def poisson_run(server, roots, budgets, modes, rate, iterations_per_poll=128, seed=0, max_seconds=600.0):
    """roots: (n, 32) uint8 host records; budgets, modes: n ints; rate: queries/s.
    Queries arrive at seeded exponential gaps (real time); the loop submits the
    arrived ones, polls the server, and records each result.  Returns a dict
    with per-query results, latency percentiles and throughput."""
    n = len(roots)
    rng = np.random.default_rng(seed)
    arrival = np.cumsum(rng.exponential(1.0 / rate, size=n)) if rate > 0 else np.zeros(n)
    results = {}
    nxt = 0
    t0 = time.perf_counter()
    while len(results) < n:
        now = time.perf_counter() - t0
        if now > max_seconds:
            raise TimeoutError(f"{len(results)} of {n} queries done after {max_seconds} s")
        while nxt < n and arrival[nxt] <= now:
            server.dvc_server_submit(roots[nxt], int(budgets[nxt]), int(modes[nxt]), nxt)
            nxt += 1
        for r in server.dvc_server_poll(iterations_per_poll):
            results[r["query_id"]] = r
        if nxt < n and not server.dvc_server_stats()["resident"]:
            time.sleep(max(0.0, min(arrival[nxt] - (time.perf_counter() - t0), 0.01)))
    wall = time.perf_counter() - t0
    lat = np.array([results[i]["t_done"] - results[i]["t_submit"] for i in range(n)])
    return {
        "results": results,
        "queries": n,
        "wall_s": wall,
        "decisions_per_s": n / wall,
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "rate": rate,
    }


def _pct(a, q):
    return float(np.percentile(np.asarray(a), q) * 1e3) if len(a) else None


class _Mover:
    """Plays the answered guesses of one poll on the games (dvc_play_move of
    each variant; the next seat draws) without blocking the serving loop: on
    a CUDA device each batch runs on its own high-priority stream with pinned
    staging and an event, and is collected once done; on the CPU (tests with
    fake contexts) it runs at once."""

    def __init__(self, ctxs, device, seed):
        import torch
        self.torch = torch
        self.ctxs = ctxs
        self.device = device
        self.seed = seed
        self.cuda = device != "cpu"
        self.stream = torch.cuda.Stream(priority=-1) if self.cuda else None
        self.pending = []
        self.batches = 0

    def submit(self, v, games, actions, states):
        torch = self.torch
        self.batches += 1
        if not self.cuda:
            st = torch.from_numpy(states.copy())
            self.ctxs[v].dvc_play_move(st, torch.tensor(actions, dtype=torch.int32), self.seed, self.batches,
                                       torch.from_numpy(games.astype(np.int32)))
            self.pending.append((None, games, st.numpy()))
            return
        hs = torch.from_numpy(states).pin_memory()
        ha = torch.tensor(actions, dtype=torch.int32).pin_memory()
        hg = torch.from_numpy(games.astype(np.int32)).pin_memory()
        out = torch.empty_like(hs).pin_memory()
        with torch.cuda.stream(self.stream):
            st = hs.to(self.device, non_blocking=True)
            act = ha.to(self.device, non_blocking=True)
            ids = hg.to(self.device, non_blocking=True)
            self.ctxs[v].dvc_play_move(st, act, self.seed, self.batches, ids, stream=self.stream)
            out.copy_(st, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        # keep the staging buffers alive until the event has passed
        self.pending.append((ev, games, out, (hs, ha, hg, st, act, ids)))

    def ready(self):
        """(games, new states) of every batch that has finished."""
        done, keep = [], []
        for p in self.pending:
            if p[0] is None or p[0].query():
                done.append((p[1], p[2] if p[0] is None else p[2].numpy()))
            else:
                keep.append(p)
        self.pending = keep
        return done


def game_serving_run(server, ctxs, n_games, rate, duration_s, budget_lo=1000, budget_hi=100000, value_frac=0.5,
                     seed=0, iterations_per_poll=256, move_seed=77, max_seconds=900.0, device="cuda"):
    """Serve move queries from n_games concurrent games of the variants of
    `ctxs` (one context per variant, game g of variant g mod len(ctxs)).

    Queries arrive at seeded exponential gaps (rate per second, real time)
    for duration_s seconds; each arrival is the next move of a game picked
    uniformly among those with no query or move outstanding, its root that
    game's current position, its budget log-uniform in [budget_lo,
    budget_hi], its mode value with probability value_frac.  When an answer
    returns, the chosen guess is played on the game (dvc_play_move of its
    variant, the next seat drawing), asynchronously; a finished game is dealt
    afresh from a reservoir of seeded deals.  After the arrival window the
    outstanding queries are drained.  Returns decisions per second over the
    whole run, latency percentiles overall, per mode and per variant, and the
    counts."""
    nv = len(ctxs)
    rng = np.random.default_rng(seed)
    variant = np.arange(n_games) % nv
    states = np.zeros((n_games, 32), dtype=np.uint8)
    reservoir = []
    for v, c in enumerate(ctxs):
        idx = np.nonzero(variant == v)[0]
        states[idx] = c.dvc_init_states(1000 + v, len(idx)).cpu().numpy()
        reservoir.append(list(c.dvc_init_states(5000 + v, max(64, len(idx))).cpu().numpy()))
    refills = [0] * nv
    names = [f"{c.cfg.nplayers}p{c.cfg.ntiles}" for c in ctxs]
    mover = _Mover(ctxs, device, move_seed)
    busy = np.zeros(n_games, dtype=bool)   # a query or a move outstanding
    idle = list(range(n_games))
    info = {}
    lat = []
    t0 = time.perf_counter()
    next_arrival = rng.exponential(1.0 / rate)
    qid = 0
    polls = 0
    moves = 0
    redeals = 0
    t_poll = t_move = t_submit = 0.0
    while True:
        now = time.perf_counter() - t0
        if now > max_seconds:
            raise TimeoutError(f"{len(lat)} queries done after {max_seconds} s")
        ts = time.perf_counter()
        while next_arrival <= min(now, duration_s) and idle:
            k = int(rng.integers(0, len(idle)))
            g = idle[k]
            idle[k] = idle[-1]
            idle.pop()
            budget = int(np.exp(rng.uniform(np.log(budget_lo), np.log(budget_hi))))
            mode = 1 if rng.random() < value_frac else 0
            server.dvc_server_submit(states[g], budget, mode, qid)
            info[qid] = (g, mode, budget)
            busy[g] = True
            qid += 1
            next_arrival += rng.exponential(1.0 / rate)
        tp = time.perf_counter()
        t_submit += tp - ts
        if now >= duration_s and not busy.any():
            break
        done = server.dvc_server_poll(iterations_per_poll) if info else []
        tm = time.perf_counter()
        t_poll += tm - tp
        polls += 1
        by_variant = {}
        for r in done:
            g, mode, budget = info.pop(r["query_id"])
            lat.append((r["t_done"] - r["t_submit"], mode, int(variant[g])))
            by_variant.setdefault(int(variant[g]), []).append((g, int(r["best_action"])))
        for v, lst in by_variant.items():
            gs = np.array([g for g, _ in lst], dtype=np.int64)
            mover.submit(v, gs, [a for _, a in lst], states[gs])
        for gs, out in mover.ready():
            over = np.nonzero(out[:, 28] != 0xFF)[0]
            for o in over:   # a finished game is dealt afresh
                v = int(variant[gs[o]])
                if not reservoir[v]:   # rare: a new batch of seeded deals
                    refills[v] += 1
                    reservoir[v] = list(ctxs[v].dvc_init_states(5000 + v + 7919 * refills[v], 256).cpu().numpy())
                out[o] = reservoir[v].pop()
                redeals += 1
            states[gs] = out
            moves += len(gs)
            busy[gs] = False
            idle.extend(int(g) for g in gs)
        t_move += time.perf_counter() - tm
        if not done and not info and now < duration_s:
            time.sleep(max(0.0, min(next_arrival - (time.perf_counter() - t0), 0.002)))
    wall = time.perf_counter() - t0
    lat_s = np.array([x[0] for x in lat])
    modes = np.array([x[1] for x in lat])
    vars_ = np.array([x[2] for x in lat])
    out = {
        "games": n_games,
        "variants": names,
        "rate": rate,
        "arrival_window_s": duration_s,
        "queries": len(lat),
        "wall_s": wall,
        "decisions_per_s": len(lat) / wall,
        "moves_played": moves,
        "games_redealt": redeals,
        "polls": polls,
        "host_s": {"poll": t_poll, "moves": t_move, "submit": t_submit},
        "p50_ms": _pct(lat_s, 50),
        "p99_ms": _pct(lat_s, 99),
        "by_mode": {},
        "by_variant": {},
    }
    for m, nm in ((0, "rollout"), (1, "value")):
        sel = lat_s[modes == m]
        out["by_mode"][nm] = {"queries": int(len(sel)), "p50_ms": _pct(sel, 50), "p99_ms": _pct(sel, 99)}
    for v, nm in enumerate(names):
        sel = lat_s[vars_ == v]
        out["by_variant"][nm] = {"queries": int(len(sel)), "p50_ms": _pct(sel, 50), "p99_ms": _pct(sel, 99)}
    return out
