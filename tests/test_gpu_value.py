"""GPU value network against the oracle: tensor-core GEMM, features, forward,
gradient, training and checkpoint resume.

Tolerances come from the arithmetic: weights are identical BF16 values on both
sides (the oracle computes in double); the GPU rounds activations to BF16
(relative 2^-9) after each of three hidden layers and accumulates in FP32, so
win probabilities agree to about 1e-2 and gradients to a few percent."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

VARIANTS = {
    "2p24": dict(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5),
    "3p24": dict(nplayers=3, ntiles=24, deal=4, max_predraw=6, max_revealed=3),
    "4p26j": dict(nplayers=4, ntiles=26, deal=3, max_predraw=8, max_revealed=3),
}


@pytest.fixture(scope="module")
def dvc():
    import paper_2403_10720_gb300 as m
    from paper_2403_10720_gb300 import build
    build.build()
    return m


def _bf16_round(x):
    return torch.as_tensor(x).to(torch.bfloat16).to(torch.float32)


@pytest.mark.parametrize("M,N,K", [(128, 512, 640), (300, 512, 512), (77, 16, 512), (256, 640, 128), (1, 32, 64)])
def test_tensor_core_gemm(dvc, M, N, K):
    ctx = dvc.Context(dvc.Config(), 0)
    g = torch.Generator().manual_seed(M * 7 + N)
    A = torch.randn((M, K), generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g)
    for act in (0, 1):
        C, Cf = ctx.dvc_gemm_bf16(A.cuda(), B.cuda(), bias.cuda(), act=act)
        torch.cuda.synchronize()
        ctx.dvc_check()
        ref = A.double() @ B.double().T + bias.double()
        err = (Cf.cpu().double() - ref).abs().max().item()
        assert err <= 1e-4 * max(1.0, ref.abs().max().item()), err
        post = torch.nn.functional.gelu(ref, approximate="tanh") if act == 1 else ref
        assert torch.allclose(C.cpu().double(), post, rtol=1e-2, atol=1e-2)


def test_gemm_output_alignment(dvc):
    """Outputs 32-byte aligned take 256-bit stores, 16-byte aligned ones
    16-byte stores: same results; an 8-byte offset is refused on the host."""
    import ctypes
    ctx = dvc.Context(dvc.Config(), 0)
    g = torch.Generator().manual_seed(11)
    M, N, K = 300, 64, 128
    A = torch.randn((M, K), generator=g).to(torch.bfloat16).cuda()
    B = torch.randn((N, K), generator=g).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).cuda()
    C0, F0 = ctx.dvc_gemm_bf16(A, B, bias, act=1)
    cbuf = torch.zeros(M * N + 16, dtype=torch.bfloat16, device="cuda")
    fbuf = torch.zeros(M * N + 8, dtype=torch.float32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = dvc.lib().dvc_gemm_bf16(ctx.h, A.data_ptr(), B.data_ptr(), bias.data_ptr(), cbuf.data_ptr() + 16,
                                 fbuf.data_ptr() + 16, M, N, K, 1, st)
    assert rc == 0
    torch.cuda.synchronize()
    ctx.dvc_check()
    assert torch.equal(cbuf[8:8 + M * N].view(M, N), C0)
    assert torch.equal(fbuf[4:4 + M * N].view(M, N), F0)
    rc = dvc.lib().dvc_gemm_bf16(ctx.h, A.data_ptr(), B.data_ptr(), bias.data_ptr(), cbuf.data_ptr() + 8,
                                 None, M, N, K, 1, st)
    assert rc == -1


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_features_exact(dvc, variant):
    kw = VARIANTS[variant]
    states = oracle.init_states(oracle.OracleConfig(**kw), 17, 200)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    got = ctx.dvc_value_features(torch.from_numpy(states).cuda()).cpu().numpy()
    for i in range(len(states)):
        assert (got[i] == oracle.value_features(states[i])).all(), i


def _net(dvc, kw, seed=5):
    ctx = dvc.Context(dvc.Config(**kw), 0)
    ctx.dvc_value_init(seed)
    p = _bf16_round(ctx.dvc_value_params().cpu())   # identical BF16 weights on both sides
    ctx.dvc_value_params(p.cuda())
    return ctx, p.numpy()


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_forward_matches_oracle(dvc, variant):
    kw = VARIANTS[variant]
    ctx, p = _net(dvc, kw)
    states = oracle.init_states(oracle.OracleConfig(**kw), 23, 300)
    got = ctx.dvc_value_eval(torch.from_numpy(states).cuda()).cpu().numpy()
    ctx.dvc_check()
    worst = 0.0
    for i in range(0, len(states), 3):
        want = oracle.value_forward(p, states[i])
        worst = max(worst, float(np.abs(got[i] - want).max()))
        assert abs(got[i].sum() - 1.0) < 1e-5
        assert (got[i][kw["nplayers"]:] == 0).all()
    assert worst < 1.5e-2, worst


def test_gradient_matches_oracle(dvc):
    kw = VARIANTS["4p26j"]
    ctx, p = _net(dvc, kw, seed=9)
    states = np.concatenate([oracle.init_states(oracle.OracleConfig(**VARIANTS[v]), 31, 40) for v in VARIANTS])
    rng = np.random.default_rng(2)
    labels = np.zeros((len(states), 4), dtype=np.float32)
    for i, s in enumerate(states):
        labels[i, :s[26]] = rng.dirichlet(np.ones(s[26]))
    loss = torch.zeros(1, device="cuda")
    ctx.dvc_value_train_step(torch.from_numpy(states).cuda(), torch.from_numpy(labels).cuda(), 0.0, loss=loss)
    g = ctx.dvc_value_grads().cpu().numpy().astype(np.float64)
    ctx.dvc_check()
    want_loss, want = oracle.value_loss_grad(p, states, labels)
    assert abs(loss.item() - want_loss) < 1e-2 * want_loss
    offs = [0, 512 * 640, 512 * 641, 512 * 641 + 512 * 512, 512 * 642 + 512 * 512, 512 * 642 + 2 * 512 * 512,
            512 * 643 + 2 * 512 * 512, 512 * 647 + 2 * 512 * 512, 855556]
    for a, b in zip(offs, offs[1:]):
        rel = np.linalg.norm(g[a:b] - want[a:b]) / max(np.linalg.norm(want[a:b]), 1e-12)
        # each gradient element sums products of BF16-rounded factors (relative
        # 2^-9 each); the first layer's passes through up to six such
        # roundings (activations, transposes, dZ of three GELU layers), so
        # sqrt(6) x 2^-9 = 4.8e-3 relative; measured 2.7e-3 to 4.5e-3 on three
        # seeds; the bound is three times the estimate
        assert rel < 1.5e-2, (a, b, rel)


def _read_checkpoint(path):
    """Version-1 value-network file: 'DVCV', u32 version, u64 count, i64 Adam
    step, then FP32 master weights, first and second moments."""
    raw = open(path, "rb").read()
    assert raw[:4] == b"DVCV"
    n = int(np.frombuffer(raw[8:16], dtype=np.uint64)[0])
    step = int(np.frombuffer(raw[16:24], dtype=np.int64)[0])
    body = np.frombuffer(raw[24:], dtype=np.float32).reshape(3, n)
    return step, body[0].astype(np.float64), body[1].astype(np.float64), body[2].astype(np.float64)


def test_adamw_update_matches_oracle(dvc, tmp_path):
    """One GPU training step's optimizer update against the oracle's AdamW in
    double, given the GPU's own gradient of that step: new master weights and
    both moments, element by element.  The GPU computes in FP32 with its
    constants rounded to FP32 (1 - b2 is then 1.3e-5 relative below 0.001,
    1 - b2^t as far off), so the bounds follow the terms of each formula:
    m = b1 m0 + (1 - b1) g to 1e-6 of |m0| + |g| (the two terms may cancel);
    v (positive terms) to 5e-5 relative; w to 2^-22 |w| plus lr times the
    update's error, i.e. m's bound over (1 - b1^t)(sqrt(vhat) + eps) and 5e-5
    of the update."""
    kw = VARIANTS["3p24"]
    ctx, _ = _net(dvc, kw, seed=5)
    states = torch.from_numpy(oracle.init_states(oracle.OracleConfig(**kw), 51, 256)).cuda()
    rng = np.random.default_rng(3)
    lab = np.zeros((256, 4), dtype=np.float32)
    lab[:, :3] = rng.dirichlet(np.ones(3), size=256)
    labels = torch.from_numpy(lab).cuda()
    lr = 2e-3
    for _ in range(4):                       # non-trivial moments first
        ctx.dvc_value_train_step(states, labels, lr)
    a, b = tmp_path / "a.dvcv", tmp_path / "b.dvcv"
    ctx.dvc_value_save(a)
    ctx.dvc_value_train_step(states, labels, lr)
    g = ctx.dvc_value_grads().cpu().numpy().astype(np.float64)
    ctx.dvc_value_save(b)
    ctx.dvc_check()
    t0, w0, m0, v0 = _read_checkpoint(a)
    t1, w1, m1, v1 = _read_checkpoint(b)
    assert t1 == t0 + 1 == 5
    ww, wm, wv = oracle.adamw_step(w0, m0, v0, g, t1, lr)
    dm = 1e-6 * (np.abs(m0) + np.abs(g)) + 1e-30
    assert (np.abs(m1 - wm) <= dm).all()
    assert (np.abs(v1 - wv) <= 5e-5 * np.abs(wv) + 1e-30).all()
    c1, c2 = 1 - 0.9 ** t1, 1 - 0.999 ** t1
    den = np.sqrt(wv / c2) + 1e-8
    upd = (wm / c1) / den
    step = np.abs(w0 - ww)
    bound = 2.0 ** -22 * np.abs(ww) + lr * (dm / c1 / den + 5e-5 * np.abs(upd)) + 1e-12
    assert (np.abs(w1 - ww) <= bound).all()
    assert (step > 0).mean() > 0.5           # the update moved most parameters


def test_training_reduces_loss_and_resumes_exactly(dvc, tmp_path):
    kw = VARIANTS["2p24"]
    ctx, _ = _net(dvc, kw, seed=3)
    states = torch.from_numpy(oracle.init_states(oracle.OracleConfig(**kw), 41, 512)).cuda()
    leaf_ids = torch.arange(512, dtype=torch.int32, device="cuda")
    wins = ctx.dvc_rollout_batch(states, 64, 5, leaf_ids, leaf_ids)
    labels = (wins.float() / 64.0).contiguous()
    # the loss cannot go below the labels' own entropy; what training removes
    # is the excess (the KL divergence from the labels)
    y = labels.cpu().double()
    entropy = float(-(y * torch.where(y > 0, y.log(), torch.zeros_like(y))).sum(1).mean())
    loss = torch.zeros(1, device="cuda")
    losses = []
    for step in range(60):
        ctx.dvc_value_train_step(states, labels, 3e-3, loss=loss)
        losses.append(loss.item())
    assert losses[-1] - entropy < 0.5 * (losses[0] - entropy), (entropy, losses[::10])
    path = tmp_path / "net.dvcv"
    ctx.dvc_value_save(path)
    for _ in range(3):
        ctx.dvc_value_train_step(states, labels, 1e-3)
    a = ctx.dvc_value_params().cpu()
    ctx2 = dvc.Context(dvc.Config(**kw), 0)
    ctx2.dvc_value_load(path)
    for _ in range(3):
        ctx2.dvc_value_train_step(states, labels, 1e-3)
    b = ctx2.dvc_value_params().cpu()
    ctx.dvc_check()
    assert torch.equal(a, b)


def test_value_mode_search(dvc):
    """MCTS with the network at the leaves: same tree mechanics (visits in
    playout units, one node per iteration), deterministic, and a finished
    leaf keeps its exact credit."""
    kw = dict(VARIANTS["3p24"], playouts=64)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    ctx.dvc_value_init(11)
    n, budget = 40, 120
    roots = ctx.dvc_init_states(8, n)
    runs = []
    for _ in range(2):
        f = dvc.Forest(ctx, roots, [budget] * n, 3)
        f.dvc_mcts_step(budget, dvc.DVC_MODE_VALUE)
        runs.append((f.dvc_root_stats().cpu(), [f.dvc_tree_export(t).cpu() for t in (0, 17)]))
    ctx.dvc_check()
    stats = runs[0][0].numpy()
    assert torch.equal(runs[0][0], runs[1][0])
    assert all(torch.equal(a, b) for a, b in zip(runs[0][1], runs[1][1]))
    assert (stats[:, 3] == budget * 64).all() and (stats[:, 6] == budget).all()
    exp = runs[0][1][0].numpy()
    nodes = exp[exp[:, 0] >= 0]
    assert len(nodes) <= budget + 1
    for a, par, vis, w in nodes[1:]:
        assert 0 <= w <= vis and vis % 64 == 0


def _zero_hidden_params(b4):
    """Every weight matrix zero: the logits are the output bias b4, so the win
    probabilities are softmax(b4) over the seats in play (relative to the
    seat to move) in closed form, the same in FP32 and in double."""
    prm = np.zeros(oracle.value_nparams(), dtype=np.float32)
    prm[-4:] = b4
    return prm


@pytest.mark.parametrize("variant,P,budgets,chains", [
    ("2p24", 32, [150, 57, 1, 0, 120, 96], 0),
    ("3p24", 16, [130, 90, 3, 64], 0),
    ("4p26j", 32, [120, 64, 100, 17, 1], 0),
    ("2p24", 8, [100] * 300, 3),
])
def test_value_mode_bit_exact(dvc, variant, P, budgets, chains):
    """Value-mode search (the network's probabilities stand in for a fresh
    leaf's playouts, each seat credited round(p * P)) against the oracle's
    value-mode search, node table for node table.  The network's hidden
    weights are zero so that p is a closed form on both sides, and b4 keeps
    every p * P at least 0.18 from a rounding tie, so FP32 on the GPU and
    double in the oracle round alike."""
    kw = dict(VARIANTS[variant], playouts=P)
    nseat = kw["nplayers"]
    b4 = np.array([0.4, -0.5, 0.0, 1.1], dtype=np.float32)
    e = np.exp(b4[:nseat].astype(np.float64))
    frac = (e / e.sum()) * P % 1.0
    assert (np.abs(frac - 0.5) > 0.18).all()
    prm = _zero_hidden_params(b4)
    ocfg = oracle.OracleConfig(**kw)
    n = len(budgets)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    ctx.dvc_value_init(1)
    ctx.dvc_value_params(torch.from_numpy(prm).cuda())
    roots = ctx.dvc_init_states(21, n)
    oroots = oracle.init_states(ocfg, 21, n)
    assert (roots.cpu().numpy() == oroots).all()
    tree_ids = np.arange(n, dtype=np.uint32) * 5 + 9
    f = dvc.Forest(ctx, roots, budgets, 8, tree_ids=tree_ids)
    if chains:
        f.dvc_forest_tune(0, 0, 0, chains)
    f.dvc_mcts_step(max(budgets), dvc.DVC_MODE_VALUE)
    stats = f.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    assert (stats[:, 6] == np.asarray(budgets)).all()
    trees = range(n) if n <= 8 else (0, 1, 149, 298, 299)
    for t in trees:
        nodes, best = oracle.mcts(ocfg, oroots[t], 8, int(tree_ids[t]), int(budgets[t]), value_params=prm)
        exp = f.dvc_tree_export(t).cpu().numpy()
        assert (exp[: len(nodes)] == nodes).all(), t
        assert (exp[len(nodes):] == -1).all(), t
        assert stats[t][0] == best[0] and stats[t][1] == best[1] and stats[t][2] == best[2], t
        assert stats[t][3] == best[3] and stats[t][5] == len(nodes), t
    f.close()
    ctx.close()


def test_value_mode_chains_agree(dvc):
    """The chained, graph-captured value pipeline gives the same trees for
    1, 3 and 8 chains, across a captured 64-iteration chunk and a tail."""
    kw = dict(VARIANTS["2p24"], playouts=16)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    ctx.dvc_value_init(13)
    n, budget = 1100, 100
    roots = ctx.dvc_init_states(27, n)
    out = []
    for chains in (1, 3, 8):
        f = dvc.Forest(ctx, roots, [budget] * n, 5)
        f.dvc_forest_tune(0, 0, 0, chains)
        f.dvc_mcts_step(70, dvc.DVC_MODE_VALUE)
        f.dvc_mcts_step(30, dvc.DVC_MODE_VALUE)
        out.append((f.dvc_root_stats().cpu(), [f.dvc_tree_export(t).cpu() for t in (0, 549, 1099)]))
        f.close()
    ctx.dvc_check()
    for stats, trees in out[1:]:
        assert torch.equal(stats, out[0][0])
        assert all(torch.equal(a, b) for a, b in zip(trees, out[0][1]))
    assert (out[0][0][:, 6] == budget).all()


def test_trained_network_gains_over_playouts(dvc):
    """After training on 131,072 states labelled by 1,024 playouts each, the
    network's win probabilities on held-out states are closer to the labels
    than a 16-playout rollout estimate, and cost less GPU time per leaf than
    the 64 playouts whose accuracy they approach."""
    from paper_2403_10720_gb300 import value_train as vt
    kw = dict(VARIANTS["2p24"], playouts=256)
    ctx = dvc.Context(dvc.Config(**kw), 0)
    ctx.dvc_value_init(1)
    states, labels = vt.make_dataset(ctx, 131072, root_seed=101)
    hs, hl = vt.make_dataset(ctx, 4096, root_seed=202)
    vt.train(ctx, states, labels, epochs=12, batch=8192, lr=1e-3)
    err_net = vt.mean_abs_error(ctx.dvc_value_eval(hs), hl, hs)
    err16 = vt.mean_abs_error(vt.rollout_estimate(ctx, hs, 16), hl, hs)
    err64 = vt.mean_abs_error(vt.rollout_estimate(ctx, hs, 64), hl, hs)
    big = ctx.dvc_init_states(303, 65536)
    ids = torch.arange(65536, dtype=torch.int32, device="cuda")
    ms_net = vt.timed(lambda: ctx.dvc_value_eval(big))
    ms64 = vt.timed(lambda: ctx.dvc_rollout_batch(big, 64, 9, ids, ids))
    print(f"held-out |dp|: net {err_net:.4f}, 16 playouts {err16:.4f}, 64 playouts {err64:.4f}; "
          f"65,536 leaves: net {ms_net:.3f} ms, 64 playouts {ms64:.3f} ms")
    assert err_net < 0.8 * err16
    assert ms_net < ms64
