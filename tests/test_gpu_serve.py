"""Serving: continuous batching of move queries, admission by memory, and
results independent of what else is resident."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

KW = dict(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5, playouts=32)


@pytest.fixture(scope="module")
def dvc():
    import paper_2403_10720_gb300 as m
    from paper_2403_10720_gb300 import build
    build.build()
    return m


def _direct(dvc, ctx, root, budget, qid, seed, mode=0):
    f = dvc.Forest(ctx, torch.from_numpy(root[None]).cuda(), [budget], seed, tree_ids=[qid])
    f.dvc_mcts_step(budget, mode)
    s = f.dvc_root_stats().cpu().numpy()[0]
    return int(s[0]), int(s[1]), int(s[2]), int(s[3])


def _key(r):
    return (r["best_action"], r["best_visits"], r["best_wins"], r["root_visits"])


def test_result_same_alone_and_in_the_mix(dvc):
    ctx = dvc.Context(dvc.Config(**KW), 0)
    roots = ctx.dvc_init_states(77, 120).cpu().numpy()
    budgets = np.random.default_rng(1).integers(20, 300, size=120)
    seed = 9
    alone = dvc.Server(ctx, 64 << 20, 512, seed=seed)
    alone.dvc_server_submit(roots[5], int(budgets[5]), 0, 5)
    res = []
    while not res:
        res = alone.dvc_server_poll(64)
    want = _key(res[0])
    assert want == _direct(dvc, ctx, roots[5], int(budgets[5]), 5, seed)
    mix = dvc.Server(ctx, 64 << 20, 512, seed=seed)
    got = {}
    order = list(range(120))
    for step in range(400):
        for i in order[step * 7:(step + 1) * 7]:       # arrivals spread over the polls
            mix.dvc_server_submit(roots[i], int(budgets[i]), 0, i)
        for r in mix.dvc_server_poll(37):
            got[r["query_id"]] = r
        if len(got) == 120:
            break
    assert len(got) == 120
    assert _key(got[5]) == want
    for i in (0, 17, 119):
        assert _key(got[i]) == _direct(dvc, ctx, roots[i], int(budgets[i]), i, seed)
    ctx.dvc_check()


def test_admission_by_memory(dvc):
    ctx = dvc.Context(dvc.Config(**KW), 0)
    roots = ctx.dvc_init_states(3, 50).cpu().numpy()
    per_slot = (1 + 640 + 4 * 256) * 36 + 2048 * 8 + 1024
    sv = dvc.Server(ctx, 10 * per_slot, 256, seed=2)
    st = sv.dvc_server_stats()
    assert 5 <= st["rollout_slots"] <= 10
    for i in range(50):
        sv.dvc_server_submit(roots[i], 200, 0, i)
    done = {}
    peak = 0
    while len(done) < 50:
        for r in sv.dvc_server_poll(64):
            done[r["query_id"]] = r
        st = sv.dvc_server_stats()
        peak = max(peak, st["resident"])
        assert st["resident"] <= st["rollout_slots"]
    assert peak == st["rollout_slots"]
    assert all(r["iterations"] == 200 and r["root_visits"] == 200 * 32 for r in done.values())


def test_value_mode_queries(dvc):
    ctx = dvc.Context(dvc.Config(**KW), 0)
    ctx.dvc_value_init(4)
    roots = ctx.dvc_init_states(8, 12).cpu().numpy()
    sv = dvc.Server(ctx, 256 << 20, 256, value_share_pct=50, seed=5)
    st = sv.dvc_server_stats()
    assert st["value_slots"] > 0 and st["rollout_slots"] > 0
    for i in range(12):
        sv.dvc_server_submit(roots[i], 100, i % 2, i)
    got = {}
    while len(got) < 12:
        for r in sv.dvc_server_poll(50):
            got[r["query_id"]] = r
    for i in (1, 3):
        assert got[i]["mode"] == 1
        assert _key(got[i]) == _direct(dvc, ctx, roots[i], 100, i, 5, mode=1)
    assert _key(got[2]) == _direct(dvc, ctx, roots[2], 100, 2, 5, mode=0)


def test_poisson_driver_reports_latency(dvc):
    from paper_2403_10720_gb300 import serving
    ctx = dvc.Context(dvc.Config(**KW), 0)
    roots = ctx.dvc_init_states(21, 200).cpu().numpy()
    budgets = np.random.default_rng(3).integers(50, 400, size=200)
    sv = dvc.Server(ctx, 512 << 20, 512, seed=3)
    out = serving.poisson_run(sv, roots, budgets, np.zeros(200, dtype=int), rate=2000.0, iterations_per_poll=64)
    assert out["queries"] == 200 and out["p99_ms"] >= out["p50_ms"] > 0
    assert all(out["results"][i]["iterations"] == budgets[i] for i in range(200))


MULTI = {
    "2p24": dict(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5, playouts=32),
    "3p24": dict(nplayers=3, ntiles=24, deal=4, max_predraw=6, max_revealed=3, playouts=32),
    "2p26": dict(nplayers=2, ntiles=26, deal=4, max_predraw=10, max_revealed=5, playouts=32),
    "4p26": dict(nplayers=4, ntiles=26, deal=3, max_predraw=8, max_revealed=3, playouts=32),
}


def test_multi_variant_mix_same_as_alone(dvc):
    """One server over four game variants, rollout and value queries mixed:
    every sampled result equals the same search run alone (its own forest of
    one tree), and a query alone in a fresh server gives the same result."""
    names = sorted(MULTI)
    ctxs = []
    for i, nm in enumerate(names):
        c = dvc.Context(dvc.Config(**MULTI[nm]), 0)
        c.dvc_value_init(40 + i)
        ctxs.append(c)
    seed = 13
    per = 24
    rng = np.random.default_rng(7)
    queries = []   # (qid, variant index, root, budget, mode)
    for vi, c in enumerate(ctxs):
        roots = c.dvc_init_states(90 + vi, per).cpu().numpy()
        for k in range(per):
            queries.append((1000 * vi + k, vi, roots[k], int(rng.integers(20, 260)), int(rng.integers(0, 2))))
    order = rng.permutation(len(queries))
    sv = dvc.Server(ctxs, 512 << 20, 512, value_share_pct=40, seed=seed)
    lanes = sv.dvc_server_lanes()
    assert len(lanes) == 2 * len(names)
    assert {(l["players"], l["tiles"], l["mode"]) for l in lanes} == {
        (MULTI[n]["nplayers"], MULTI[n]["ntiles"], m) for n in names for m in (0, 1)}
    got = {}
    for step in range(2000):
        for j in order[step * 9:(step + 1) * 9]:
            qid, vi, root, b, mode = queries[j]
            sv.dvc_server_submit(root, b, mode, qid)
        for r in sv.dvc_server_poll(41):
            got[r["query_id"]] = r
        if len(got) == len(queries):
            break
    assert len(got) == len(queries)
    for c in ctxs:
        c.dvc_check()
    for qid, vi, root, b, mode in queries[::5]:
        r = got[qid]
        assert r["mode"] == mode and r["iterations"] == b
        assert _key(r) == _direct(dvc, ctxs[vi], root, b, qid, seed, mode=mode), (qid, vi, mode)
    # alone in a fresh single-variant server
    qid, vi, root, b, mode = next(q for q in queries if q[1] == 3 and q[4] == 1)
    alone = dvc.Server(ctxs[vi], 64 << 20, 512, value_share_pct=50, seed=seed)
    alone.dvc_server_submit(root, b, mode, qid)
    res = []
    while not res:
        res = alone.dvc_server_poll(64)
    assert _key(res[0]) == _key(got[qid])
    # a root of a variant the server does not hold is refused on the host
    other = dvc.Context(dvc.Config(nplayers=4, ntiles=24, deal=3, playouts=32), 0)
    r4 = other.dvc_init_states(1, 1).cpu().numpy()[0]
    with pytest.raises(dvc.DvcError):
        sv.dvc_server_submit(r4, 100, 0, 99999)
    sv.close()
    alone.close()
