"""Failure paths of the library, each reached safely: host-side refusals
before anything is enqueued, a device allocation that fails cleanly, and
errors that kernels latch and dvc_check reports.  After each failure the
context keeps working."""
import numpy as np
import pytest
import torch

from statefmt import encode

pytestmark = pytest.mark.gpu

KW2 = dict(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5, playouts=16)
KW4 = dict(nplayers=4, ntiles=26, deal=3, max_predraw=8, max_revealed=3, playouts=16)
E_INVALID, E_OOM, E_UNSUPPORTED = -1, -2, -5


@pytest.fixture(scope="module")
def dvc():
    import paper_2403_10720_gb300 as m
    from paper_2403_10720_gb300 import build
    build.build()
    return m


def _code(exc):
    return exc.value.code


def _still_works(dvc, ctx, kw=KW2):
    roots = ctx.dvc_init_states(5, 3)
    f = dvc.Forest(ctx, roots, [40, 40, 40], 1)
    f.dvc_mcts_step(40)
    st = f.dvc_root_stats().cpu().numpy()
    ctx.dvc_check()
    assert (st[:, 6] == 40).all() and (st[:, 3] == 40 * kw["playouts"]).all()
    f.close()


def _oversized_view():
    """A 4-player, 26-tile view whose counting table needs 35,328 cells, over
    the 32,768 a context holds: the seat to move holds two numbered tiles,
    each opponent seven face-down tiles with no face-up anchor, both jokers
    unseen: (2 + 1) x (7 + 1)^3 cells per layer over 23 layers."""
    own = [0, 1]
    rest = [t for t in range(26) if t not in own]
    rng = np.random.default_rng(8)
    rng.shuffle(rest)
    hands = [own] + [sorted(rest[7 * k:7 * k + 7], key=lambda t: (t >= 24, t)) for k in range(3)]
    return encode(hands, set(), cur=0, drawn=None, ntiles=26)


def test_server_budget_below_one_slot_is_oom(dvc):
    ctx = dvc.Context(dvc.Config(**KW2), 0)
    with pytest.raises(dvc.DvcError) as e:
        dvc.Server(ctx, 1000, 1000)
    assert _code(e) == E_OOM
    _still_works(dvc, ctx)


def test_forest_arena_that_cannot_be_allocated_is_oom(dvc):
    # 1,024 trees of 2^24 iterations need about 3.3 TB of node arena: the
    # device allocation fails cleanly and the forest is not created
    ctx = dvc.Context(dvc.Config(**KW2), 0)
    roots = ctx.dvc_init_states(1, 1024)
    with pytest.raises(dvc.DvcError) as e:
        dvc.Forest(ctx, roots, [1 << 24] * 1024, 1)
    assert _code(e) == E_OOM
    _still_works(dvc, ctx)


def test_view_over_table_capacity_is_unsupported(dvc):
    ctx = dvc.Context(dvc.Config(**KW4), 0)
    roots = ctx.dvc_init_states(3, 4)
    roots[2] = torch.from_numpy(_oversized_view()).cuda()
    ids = torch.arange(4, dtype=torch.int32, device="cuda")
    out = ctx.dvc_determinize(roots, -1, 7, ids, ids)
    torch.cuda.synchronize()
    assert torch.equal(out[2], roots[2])               # that output is the root itself
    with pytest.raises(dvc.DvcError) as e:
        ctx.dvc_check()
    assert _code(e) == E_UNSUPPORTED
    ctx.dvc_check()                                     # reported once, then cleared
    # in a forest: that tree runs no iteration, the others search normally
    f = dvc.Forest(ctx, roots, [30, 30, 30, 30], 2)
    f.dvc_mcts_step(30)
    st = f.dvc_root_stats().cpu().numpy()
    with pytest.raises(dvc.DvcError) as e:
        ctx.dvc_check()
    assert _code(e) == E_UNSUPPORTED
    assert st[2, 6] == 0 and (st[[0, 1, 3], 6] == 30).all()
    f.close()
    _still_works(dvc, ctx, KW4)


def test_root_of_another_variant_in_a_forest_is_invalid(dvc):
    ctx = dvc.Context(dvc.Config(**KW2), 0)
    other = dvc.Context(dvc.Config(**KW4), 0)
    roots = ctx.dvc_init_states(4, 3)
    roots[1] = other.dvc_init_states(4, 1)[0]
    f = dvc.Forest(ctx, roots, [20, 20, 20], 3)
    f.dvc_mcts_step(20)
    st = f.dvc_root_stats().cpu().numpy()
    with pytest.raises(dvc.DvcError) as e:
        ctx.dvc_check()
    assert _code(e) == E_INVALID
    assert st[1, 6] == 0 and st[0, 6] == 20 and st[2, 6] == 20
    f.close()
    _still_works(dvc, ctx)


def test_host_refusals_enqueue_nothing(dvc):
    ctx = dvc.Context(dvc.Config(**KW2), 0)
    roots = ctx.dvc_init_states(6, 4)
    ids = torch.arange(4, dtype=torch.int32, device="cuda")
    # host memory where device memory is needed (the binding refuses host
    # tensors itself, so call the C ABI directly)
    host = roots.cpu().pin_memory()
    out = torch.zeros_like(roots)
    rc = dvc.lib().dvc_determinize(ctx.h, host.data_ptr(), 4, -1, 1, ids.data_ptr(), ids.data_ptr(),
                                   out.data_ptr(), None)
    assert rc == E_INVALID
    torch.cuda.synchronize()
    assert int(out.abs().max()) == 0
    with pytest.raises(dvc.DvcError) as e:            # output overlapping the input
        ctx.dvc_determinize(roots, -1, 1, ids, ids, out=roots)
    assert _code(e) == E_INVALID
    with pytest.raises(dvc.DvcError) as e:            # observer outside the game
        ctx.dvc_determinize(roots, 2, 1, ids, ids)
    assert _code(e) == E_INVALID
    with pytest.raises(dvc.DvcError) as e:            # budgets outside 0..2^24
        dvc.Forest(ctx, roots, [10, -1, 10, 10], 1)
    assert _code(e) == E_INVALID
    sv = dvc.Server(ctx, 64 << 20, 100)
    with pytest.raises(dvc.DvcError) as e:            # budget above the server's maximum
        sv.dvc_server_submit(roots[0].cpu().numpy(), 101, 0, 1)
    assert _code(e) == E_INVALID
    with pytest.raises(dvc.DvcError) as e:            # value mode without value slots
        sv.dvc_server_submit(roots[0].cpu().numpy(), 50, 1, 2)
    assert _code(e) == E_UNSUPPORTED
    sv.close()
    _still_works(dvc, ctx)


def test_gemm_wait_runs_out_and_reports_timeout(dvc):
    """The GEMM's mbarrier waits are bounded: with its copy-issuing warp
    issuing nothing (the test hook), the other warps' waits run out after
    20 ms with nothing in flight, the kernel frees its tensor memory and
    exits, and dvc_check reports DVC_E_TIMEOUT.  The GEMM works afterwards."""
    ctx = dvc.Context(dvc.Config(**KW2), 0)
    g = torch.Generator().manual_seed(3)
    A = torch.randn((128, 64), generator=g).to(torch.bfloat16).cuda()
    B = torch.randn((16, 64), generator=g).to(torch.bfloat16).cuda()
    Cf = torch.full((128, 16), 7.0, device="cuda")
    rc = dvc.lib().dvc_gemm_timeout_probe(ctx.h, A.data_ptr(), B.data_ptr(), Cf.data_ptr(), 128, 16, 64, 20, None)
    assert rc == 0
    with pytest.raises(dvc.DvcError) as e:
        ctx.dvc_check()
    assert _code(e) == -4                               # DVC_E_TIMEOUT
    assert bool((Cf == 7.0).all())                      # nothing written
    _, out = ctx.dvc_gemm_bf16(A, B, None, act=0)
    torch.cuda.synchronize()
    ctx.dvc_check()
    ref = A.double().cpu() @ B.double().cpu().T
    assert (out.cpu().double() - ref).abs().max().item() < 1e-3
