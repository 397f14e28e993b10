"""dvc_determinize_noalloc: the determinizer for callers that cannot allocate
device memory (memory fully held by another framework's caching allocator, or
a process that may not allocate after start-up).  Its scratch is a fixed
device array inside the library, so its results must equal those of
dvc_determinize, which works in a context's allocated workspace.

Kept in its own file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest
import torch

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
