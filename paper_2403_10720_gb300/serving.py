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
