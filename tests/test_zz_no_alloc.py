"""dvc_determinize_noalloc: the determinizer for callers that cannot allocate
device memory (memory fully held by another framework's caching allocator, or
a process that may not allocate after start-up).  Its scratch is a fixed
device array inside the library, so its results must equal those of
dvc_determinize, which works in a context's allocated workspace.

Kept in its own file that pytest collects last.
"""
import ctypes
import os
import sys

import numpy as np
import pytest
import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from statefmt import encode  # noqa: E402

pytestmark = pytest.mark.gpu


def _u32(a):
    return torch.from_numpy(np.asarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _call(L, roots, observer, seed, tids, iids, out, status):
    return L.dvc_determinize_noalloc(ctypes.c_void_p(roots.data_ptr()), roots.shape[0], observer, seed,
                                     ctypes.c_void_p(tids.data_ptr()), ctypes.c_void_p(iids.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_determinize_matches_allocating_entry_point():
    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build
    build.build()
    L = dvc.lib()
    cases = [  # two calls in a row, different variants, so the second sees the first's leftovers
        (dict(nplayers=4, ntiles=26, deal=3, max_predraw=8, max_revealed=3), 41, 64),
        (dict(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5), 42, 37),
    ]
    for kw, seed, n in cases:
        ctx = dvc.Context(dvc.Config(**kw), 0)
        roots = ctx.dvc_init_states(seed, n)
        rng = np.random.default_rng(seed)
        tids = _u32(rng.integers(0, 1 << 30, size=n))
        iids = _u32(rng.integers(0, 1 << 30, size=n))
        want = ctx.dvc_determinize(roots, -1, seed * 7, tids, iids)
        got = torch.zeros_like(roots)
        status = torch.full((n,), -99, dtype=torch.int32, device="cuda")
        assert _call(L, roots, -1, seed * 7, tids, iids, got, status) == 0
        torch.cuda.synchronize()
        ctx.dvc_check()
        assert (status == 0).all()
        assert torch.equal(got, want)           # bit-exact, like every parity test here
        ctx.close()


def test_noalloc_rejects_more_roots_than_its_scratch_holds():
    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build
    build.build()
    L = dvc.lib()
    n = 65
    roots = torch.zeros((n, 32), dtype=torch.uint8, device="cuda")
    out = torch.full((n, 32), 7, dtype=torch.uint8, device="cuda")
    ids = torch.zeros(n, dtype=torch.int32, device="cuda")
    status = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert _call(L, roots, -1, 1, ids, ids, out, status) == -5   # DVC_E_UNSUPPORTED, nothing enqueued
    torch.cuda.synchronize()
    assert int(out.min()) == 7 and int(out.max()) == 7


def _big_view():
    """A 4-player, 26-tile view whose counting table needs more than 16,384
    cells: the observer holds two numbered tiles, each opponent six face-down
    tiles with no face-up anchor, both jokers unseen.  Cells = (jokers + 1) x
    (6 + 1)^3 per layer over 22 + 1 layers = 23,667 (the context path holds
    up to 32,768)."""
    own = [0, 1]
    rest = [t for t in range(26) if t not in own]
    rng = np.random.default_rng(5)
    rng.shuffle(rest)
    hands = [own] + [sorted(rest[6 * k:6 * k + 6], key=lambda t: (t >= 24, t)) for k in range(3)]
    return encode(hands, set(), cur=0, drawn=None, ntiles=26)


def test_noalloc_per_root_status_for_oversized_view_and_bad_observer():
    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build
    build.build()
    L = dvc.lib()
    ctx = dvc.Context(dvc.Config(nplayers=4, ntiles=26, deal=3, max_predraw=8, max_revealed=3), 0)
    n, big = 9, 5
    roots = ctx.dvc_init_states(43, n)
    roots[big] = torch.from_numpy(_big_view()).cuda()
    tids = _u32(np.arange(n) + 100)
    iids = _u32(np.arange(n) * 3)
    want = ctx.dvc_determinize(roots, -1, 11, tids, iids)
    got = torch.zeros_like(roots)
    status = torch.full((n,), -99, dtype=torch.int32, device="cuda")
    assert _call(L, roots, -1, 11, tids, iids, got, status) == 0
    torch.cuda.synchronize()
    ctx.dvc_check()
    st = status.cpu().tolist()
    assert st[big] == -5                                  # DVC_E_UNSUPPORTED: table over 16,384 cells
    assert torch.equal(got[big], roots[big])              # that output is the root itself
    keep = [i for i in range(n) if i != big]
    assert all(st[i] == 0 for i in keep)
    assert torch.equal(got[keep], want[keep])
    ctx.close()
    # a 2-player root asked for seat 3's view: per-root DVC_E_INVALID, output = root
    ctx2 = dvc.Context(dvc.Config(nplayers=2, ntiles=24, deal=4, max_predraw=10, max_revealed=5), 0)
    roots2 = ctx2.dvc_init_states(44, 4)
    ids = _u32(np.arange(4))
    got2 = torch.zeros_like(roots2)
    status2 = torch.full((4,), -99, dtype=torch.int32, device="cuda")
    assert _call(L, roots2, 3, 1, ids, ids, got2, status2) == 0
    torch.cuda.synchronize()
    assert status2.cpu().tolist() == [-1] * 4
    assert torch.equal(got2, roots2)
    ctx2.close()


def test_noalloc_refuses_overlap_and_host_memory_before_enqueueing():
    import paper_2403_10720_gb300 as dvc
    from paper_2403_10720_gb300 import build
    build.build()
    L = dvc.lib()
    n = 8
    buf = torch.zeros((2 * n, 32), dtype=torch.uint8, device="cuda")
    ids = torch.zeros(n, dtype=torch.int32, device="cuda")
    status = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    # output starting inside the input range
    assert _call(L, buf[:n], -1, 1, ids, ids, buf[n // 2:n // 2 + n], status) == -1
    # pinned and pageable host memory are not memory of the current device
    pinned = torch.zeros((n, 32), dtype=torch.uint8).pin_memory()
    assert _call(L, pinned, -1, 1, ids, ids, buf[n:], status) == -1
    pageable = torch.zeros((n, 32), dtype=torch.uint8)
    assert _call(L, buf[:n], -1, 1, ids, ids, pageable, status) == -1
    torch.cuda.synchronize()
    assert int(status.min()) == 7 and int(status.max()) == 7   # nothing ran
