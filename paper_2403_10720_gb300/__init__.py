"""Python binding of libdvc (include/dvc.h): a GB300 engine for the Da Vinci
Code Monte Carlo Tree Search of arXiv 2403.10720.

Argument marshalling only.  Every step of the method runs in the CUDA library;
this module passes torch tensors' device pointers and the current stream.
Importing it loads libdvc.so from this directory and fails loudly if the
library is missing: there is no CPU fallback.

Names follow the C ABI (dvc_create, dvc_init_states, dvc_rollout_batch, ...).
Game states are torch.uint8 CUDA tensors of shape (n, 32) in the dvc_state
layout.  `Context` and `Forest` own the C handles and free them.
"""
import ctypes
import os
import re
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdvc.so")

DVC_OK = 0
DVC_MODE_ROLLOUT = 0
DVC_MODE_VALUE = 1
ERRORS = {-1: "DVC_E_INVALID", -2: "DVC_E_OOM", -3: "DVC_E_CUDA", -4: "DVC_E_TIMEOUT", -5: "DVC_E_UNSUPPORTED",
          -6: "DVC_E_INTERNAL"}


class DvcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class dvc_config(ctypes.Structure):
    _fields_ = [
        ("nplayers", ctypes.c_int32),
        ("ntiles", ctypes.c_int32),
        ("deal", ctypes.c_int32),
        ("max_predraw", ctypes.c_int32),
        ("max_revealed", ctypes.c_int32),
        ("cont_thr", ctypes.c_uint32),
        ("c_uct", ctypes.c_double),
        ("d_max", ctypes.c_int32),
        ("playouts", ctypes.c_int32),
        ("policy", ctypes.c_int32),
        ("tree_continue", ctypes.c_int32),
        ("vanilla", ctypes.c_int32),
    ]


@dataclass
class Config:
    """Game and search parameters (see dvc_config in include/dvc.h)."""
    nplayers: int = 2
    ntiles: int = 24
    deal: int = 4
    max_predraw: int = 0
    max_revealed: int = 5
    cont_thr: int = 1 << 31
    c_uct: float = 1.4142135623730951
    d_max: int = 8
    playouts: int = 1
    policy: int = 0  # playout guesses: 0 uniform, 1 ordering-aware
    tree_continue: int = 0  # 1: the full game tree (a correct in-tree guess keeps the turn)
    vanilla: int = 0  # 1: the root's children are plausible-number sets (vanilla MCTS-dvc)

    def c(self) -> dvc_config:
        return dvc_config(self.nplayers, self.ntiles, self.deal, self.max_predraw, self.max_revealed,
                          self.cont_thr, self.c_uct, self.d_max, self.playouts, self.policy, self.tree_continue,
                          self.vanilla)


class dvc_result(ctypes.Structure):
    _fields_ = [
        ("query_id", ctypes.c_uint64),
        ("best_action", ctypes.c_int32),
        ("best_visits", ctypes.c_int32),
        ("best_wins", ctypes.c_int32),
        ("root_visits", ctypes.c_int32),
        ("iterations", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("t_submit", ctypes.c_double),
        ("t_done", ctypes.c_double),
    ]


_lib = None


def lib():
    """The loaded libdvc.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdvc.so not built at {LIB_PATH}; run paper_2403_10720_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u32, u64, i = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "dvc_create": ([ctypes.POINTER(vp), ctypes.POINTER(dvc_config), i], i),
            "dvc_destroy": ([vp], None),
            "dvc_last_error": ([vp], ctypes.c_char_p),
            "dvc_check": ([vp], i),
            "dvc_init_states": ([vp, u64, i, vp, vp], i),
            "dvc_determinize": ([vp, vp, i, i, u64, vp, vp, vp, vp], i),
            "dvc_rollout_batch": ([vp, vp, i, i, u64, vp, vp, vp, vp, vp], i),
            "dvc_play_move": ([vp, vp, i, vp, u64, vp, u32, vp], i),
            "dvc_forest_create": ([vp, i, vp, vp, vp, u64, ctypes.POINTER(vp), vp], i),
            "dvc_forest_destroy": ([vp], None),
            "dvc_forest_reset": ([vp, vp, vp], i),
            "dvc_forest_tune": ([vp, i, i, i, i], i),
            "dvc_mcts_step": ([vp, i, i, vp], i),
            "dvc_mcts_select": ([vp, vp], i),
            "dvc_mcts_expand": ([vp, vp], i),
            "dvc_mcts_backprop": ([vp, vp, vp], i),
            "dvc_forest_leaves": ([vp, pp, pp, pp], i),
            "dvc_root_stats": ([vp, vp, vp], i),
            "dvc_forest_counters": ([vp, vp, vp], i),
            "dvc_forest_work": ([vp, vp, vp], i),
            "dvc_forest_count_work": ([vp, i], i),
            "dvc_forest_order": ([vp, vp, i], i),
            "dvc_root_merge": ([vp, i, vp, vp], i),
            "dvc_forest_compaction": ([vp, i, i], i),
            "dvc_tree_export": ([vp, i, vp, vp], i),
            "dvc_philox": ([vp, i, vp, vp, vp, i, vp], i),
            "dvc_determinize_noalloc": ([vp, i, i, u64, vp, vp, vp, vp, vp], i),
            "dvc_value_init": ([vp, u64, vp], i),
            "dvc_value_params": ([vp, vp, i, vp], i),
            "dvc_value_features": ([vp, vp, i, vp, vp], i),
            "dvc_value_eval": ([vp, vp, i, vp, vp], i),
            "dvc_value_train_step": ([vp, vp, vp, i, ctypes.c_float, vp, vp], i),
            "dvc_value_grads": ([vp, vp, vp], i),
            "dvc_value_save": ([vp, ctypes.c_char_p], i),
            "dvc_value_load": ([vp, ctypes.c_char_p], i),
            "dvc_gemm_bf16": ([vp, vp, vp, vp, vp, vp, i, i, i, i, vp], i),
            "dvc_gemm_timeout_probe": ([vp, vp, vp, vp, i, i, i, i, vp], i),
            "dvc_server_create": ([vp, ctypes.c_size_t, i, i, u64, ctypes.POINTER(vp)], i),
            "dvc_server_destroy": ([vp], None),
            "dvc_server_submit": ([vp, vp, i, i, u64], i),
            "dvc_server_poll": ([vp, i, ctypes.POINTER(dvc_result), i], i),
            "dvc_server_stats": ([vp, ctypes.POINTER(ctypes.c_int64)], i),
            "dvc_server_create_multi": ([ctypes.POINTER(vp), i, vp, ctypes.c_size_t, i, i, u64,
                                         ctypes.POINTER(vp)], i),
            "dvc_server_lanes": ([vp, i, ctypes.POINTER(ctypes.c_int32)], i),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def declared_symbols(header=None):
    """Function names declared in include/dvc.h."""
    header = header or os.path.join(os.path.dirname(_HERE), "include", "dvc.h")
    text = open(header).read()
    return sorted(set(re.findall(r"\b(dvc_[a-z0-9_]+)\s*\(", text)))


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """Owns a dvc_ctx (dvc_create / dvc_destroy)."""

    def __init__(self, cfg: Config, device: int = 0):
        self.cfg = cfg
        self.device = device
        h = ctypes.c_void_p()
        c = cfg.c()
        rc = lib().dvc_create(ctypes.byref(h), ctypes.byref(c), device)
        if rc:
            raise DvcError(rc, "dvc_create")
        self.h = h

    def _rc(self, rc, what):
        if rc:
            raise DvcError(rc, f"{what}: {lib().dvc_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            lib().dvc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dev(self):
        return torch.device("cuda", self.device)

    # --- entry points -------------------------------------------------------
    def dvc_check(self):
        self._rc(lib().dvc_check(self.h), "dvc_check")

    def dvc_init_states(self, seed, n, out=None, stream=None):
        out = torch.empty((n, 32), dtype=torch.uint8, device=self.dev()) if out is None else out
        self._rc(lib().dvc_init_states(self.h, seed, n, _ptr(out), _stream(stream)), "dvc_init_states")
        return out

    def dvc_determinize(self, roots, observer, seed, tree_ids, iter_ids, out=None, stream=None):
        n = roots.shape[0]
        out = torch.empty_like(roots) if out is None else out
        self._rc(lib().dvc_determinize(self.h, _ptr(roots), n, observer, seed, _ptr(tree_ids), _ptr(iter_ids),
                                       _ptr(out), _stream(stream)), "dvc_determinize")
        return out

    def dvc_rollout_batch(self, leaves, playouts, seed, tree_ids, leaf_ids, wins=None, words=None, stream=None):
        n = leaves.shape[0]
        wins = torch.empty((n, 4), dtype=torch.int32, device=self.dev()) if wins is None else wins
        self._rc(lib().dvc_rollout_batch(self.h, _ptr(leaves), n, playouts, seed, _ptr(tree_ids), _ptr(leaf_ids),
                                         _ptr(wins), _ptr(words), _stream(stream)), "dvc_rollout_batch")
        return wins

    def dvc_play_move(self, states, actions, seed, turn, game_ids=None, stream=None):
        """One self-play move per game, in place on `states` (n x 32 uint8);
        actions: n int32 action codes, -1 = no move."""
        self._rc(lib().dvc_play_move(self.h, _ptr(states), states.shape[0], _ptr(actions), seed, _ptr(game_ids),
                                     turn, _stream(stream)), "dvc_play_move")
        return states

    VALUE_NPARAMS = 855556

    def dvc_value_init(self, seed, stream=None):
        self._rc(lib().dvc_value_init(self.h, seed, _stream(stream)), "dvc_value_init")

    def dvc_value_params(self, params=None, stream=None):
        """Without `params`: returns the FP32 parameters; with: loads them."""
        if params is None:
            out = torch.empty(self.VALUE_NPARAMS, dtype=torch.float32, device=self.dev())
            self._rc(lib().dvc_value_params(self.h, _ptr(out), 0, _stream(stream)), "dvc_value_params")
            return out
        self._rc(lib().dvc_value_params(self.h, _ptr(params), 1, _stream(stream)), "dvc_value_params")
        return params

    def dvc_value_features(self, states, stream=None):
        out = torch.empty((states.shape[0], 640), dtype=torch.float32, device=self.dev())
        self._rc(lib().dvc_value_features(self.h, _ptr(states), states.shape[0], _ptr(out), _stream(stream)),
                 "dvc_value_features")
        return out

    def dvc_value_eval(self, leaves, out=None, stream=None):
        out = torch.empty((leaves.shape[0], 4), dtype=torch.float32, device=self.dev()) if out is None else out
        self._rc(lib().dvc_value_eval(self.h, _ptr(leaves), leaves.shape[0], _ptr(out), _stream(stream)),
                 "dvc_value_eval")
        return out

    def dvc_value_train_step(self, states, labels, lr, loss=None, stream=None):
        self._rc(lib().dvc_value_train_step(self.h, _ptr(states), _ptr(labels), states.shape[0], lr, _ptr(loss),
                                            _stream(stream)), "dvc_value_train_step")
        return loss

    def dvc_value_grads(self, stream=None):
        out = torch.empty(self.VALUE_NPARAMS, dtype=torch.float32, device=self.dev())
        self._rc(lib().dvc_value_grads(self.h, _ptr(out), _stream(stream)), "dvc_value_grads")
        return out

    def dvc_value_save(self, path):
        self._rc(lib().dvc_value_save(self.h, str(path).encode()), "dvc_value_save")

    def dvc_value_load(self, path):
        self._rc(lib().dvc_value_load(self.h, str(path).encode()), "dvc_value_load")

    def dvc_gemm_bf16(self, A, B, bias=None, act=0, want_bf16=True, want_f32=True, stream=None):
        M, K = A.shape
        N = B.shape[0]
        C = torch.empty((M, N), dtype=torch.bfloat16, device=self.dev()) if want_bf16 else None
        Cf = torch.empty((M, N), dtype=torch.float32, device=self.dev()) if want_f32 else None
        self._rc(lib().dvc_gemm_bf16(self.h, _ptr(A), _ptr(B), _ptr(bias), _ptr(C), _ptr(Cf), M, N, K, act,
                                     _stream(stream)), "dvc_gemm_bf16")
        return C, Cf

    def dvc_philox(self, ctr, key, use_reference=False, stream=None):
        n = ctr.shape[0]
        out = torch.empty((n, 4), dtype=torch.int32, device=self.dev())
        self._rc(lib().dvc_philox(self.h, n, _ptr(ctr), _ptr(key), _ptr(out), int(use_reference),
                                  _stream(stream)), "dvc_philox")
        return out


class Forest:
    """Owns a dvc_forest (dvc_forest_create / dvc_forest_destroy)."""

    def __init__(self, ctx: Context, roots, budgets, seed, tree_ids=None, stream=None):
        import numpy as np
        self.ctx = ctx
        self.n = roots.shape[0]
        self.budgets = np.ascontiguousarray(np.asarray(budgets, dtype=np.int32).reshape(self.n))
        tid = None
        if tree_ids is not None:
            self._tid = np.ascontiguousarray(np.asarray(tree_ids, dtype=np.uint32).reshape(self.n))
            tid = self._tid.ctypes.data_as(ctypes.c_void_p)
        h = ctypes.c_void_p()
        ctx._rc(lib().dvc_forest_create(ctx.h, self.n, _ptr(roots), self.budgets.ctypes.data_as(ctypes.c_void_p),
                                        tid, seed, ctypes.byref(h), _stream(stream)), "dvc_forest_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().dvc_forest_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dvc_forest_tune(self, engine=0, trees_per_cta=0, warps_per_cta=0, chains=0):
        self.ctx._rc(lib().dvc_forest_tune(self.h, engine, trees_per_cta, warps_per_cta, chains), "dvc_forest_tune")

    def dvc_forest_reset(self, roots=None, stream=None):
        self.ctx._rc(lib().dvc_forest_reset(self.h, _ptr(roots), _stream(stream)), "dvc_forest_reset")

    def dvc_mcts_step(self, n_iterations, mode=DVC_MODE_ROLLOUT, stream=None):
        self.ctx._rc(lib().dvc_mcts_step(self.h, n_iterations, mode, _stream(stream)), "dvc_mcts_step")

    def dvc_mcts_select(self, stream=None):
        self.ctx._rc(lib().dvc_mcts_select(self.h, _stream(stream)), "dvc_mcts_select")

    def dvc_mcts_expand(self, stream=None):
        self.ctx._rc(lib().dvc_mcts_expand(self.h, _stream(stream)), "dvc_mcts_expand")

    def dvc_mcts_backprop(self, wins, stream=None):
        self.ctx._rc(lib().dvc_mcts_backprop(self.h, _ptr(wins), _stream(stream)), "dvc_mcts_backprop")

    def dvc_forest_leaves(self):
        """Raw device pointers (leaves, tree ids, leaf ids) owned by the forest."""
        a, b, c = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        self.ctx._rc(lib().dvc_forest_leaves(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
                     "dvc_forest_leaves")
        return a.value, b.value, c.value

    def dvc_forest_counters(self, out=None, stream=None):
        out = torch.zeros(1, dtype=torch.int64, device=self.ctx.dev()) if out is None else out
        self.ctx._rc(lib().dvc_forest_counters(self.h, _ptr(out), _stream(stream)), "dvc_forest_counters")
        return out

    def dvc_forest_compaction(self, receivers, donate_at=8):
        self.ctx._rc(lib().dvc_forest_compaction(self.h, receivers, donate_at), "dvc_forest_compaction")

    def dvc_root_merge(self, K, out=None, stream=None):
        """Root-parallel merge over groups of K consecutive trees: (n / K, 8) int32."""
        out = torch.empty((self.n // K, 8), dtype=torch.int32, device=self.ctx.dev()) if out is None else out
        self.ctx._rc(lib().dvc_root_merge(self.h, K, _ptr(out), _stream(stream)), "dvc_root_merge")
        return out

    def dvc_forest_order(self, order, n_active=0):
        """Trees per CTA by a caller's permutation; the fused engine runs the first n_active (0 = all).
        order None restores the default order."""
        if order is None:
            self.ctx._rc(lib().dvc_forest_order(self.h, None, 0), "dvc_forest_order")
            return
        import numpy as np
        o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
        if o.shape != (self.n,):
            raise ValueError("order must hold one entry per tree")
        self.ctx._rc(lib().dvc_forest_order(self.h, o.ctypes.data_as(ctypes.c_void_p), int(n_active)),
                     "dvc_forest_order")

    def dvc_forest_count_work(self, on):
        """Keep (True, the default) or skip the work counters in the playout kernels."""
        self.ctx._rc(lib().dvc_forest_count_work(self.h, 1 if on else 0), "dvc_forest_count_work")

    def dvc_forest_work(self, out=None, stream=None):
        """(random words, game steps) of the forest's playouts since the last call."""
        out = torch.zeros(2, dtype=torch.int64, device=self.ctx.dev()) if out is None else out
        self.ctx._rc(lib().dvc_forest_work(self.h, _ptr(out), _stream(stream)), "dvc_forest_work")
        return out

    def dvc_root_stats(self, out=None, stream=None):
        out = torch.empty((self.n, 8), dtype=torch.int32, device=self.ctx.dev()) if out is None else out
        self.ctx._rc(lib().dvc_root_stats(self.h, _ptr(out), _stream(stream)), "dvc_root_stats")
        return out

    def dvc_tree_export(self, tree, stream=None):
        rows = int(self.budgets[tree]) + 1
        out = torch.empty((rows, 4), dtype=torch.int32, device=self.ctx.dev())
        self.ctx._rc(lib().dvc_tree_export(self.h, tree, _ptr(out), _stream(stream)), "dvc_tree_export")
        return out


class Server:
    """Owns a dvc_server: continuous batching of move queries (see include/dvc.h).
    `ctx` is one Context, or a list of Contexts of distinct game variants that
    share the HBM budget (by `weights`, equal if None)."""

    def __init__(self, ctx, hbm_budget: int, max_budget: int, value_share_pct: int = 0, seed: int = 1,
                 weights=None):
        ctxs = list(ctx) if isinstance(ctx, (list, tuple)) else [ctx]
        self.ctxs = ctxs
        self.ctx = ctxs[0]
        h = ctypes.c_void_p()
        if len(ctxs) == 1 and weights is None:
            rc = lib().dvc_server_create(self.ctx.h, hbm_budget, max_budget, value_share_pct, seed, ctypes.byref(h))
        else:
            arr = (ctypes.c_void_p * len(ctxs))(*[c.h.value for c in ctxs])
            w = None
            if weights is not None:
                self._w = (ctypes.c_int32 * len(ctxs))(*[int(x) for x in weights])
                w = ctypes.cast(self._w, ctypes.c_void_p)
            rc = lib().dvc_server_create_multi(arr, len(ctxs), w, hbm_budget, max_budget, value_share_pct, seed,
                                               ctypes.byref(h))
        self.ctx._rc(rc, "dvc_server_create")
        self.h = h
        self._buf = (dvc_result * 65536)()

    def close(self):
        if getattr(self, "h", None):
            lib().dvc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dvc_server_submit(self, root, budget, mode, query_id):
        import numpy as np
        r = np.ascontiguousarray(np.asarray(root, dtype=np.uint8).reshape(32))
        self.ctx._rc(lib().dvc_server_submit(self.h, r.ctypes.data_as(ctypes.c_void_p), budget, mode, query_id),
                     "dvc_server_submit")

    def dvc_server_poll(self, iterations):
        n = lib().dvc_server_poll(self.h, iterations, self._buf, len(self._buf))
        if n < 0:
            self.ctx._rc(n, "dvc_server_poll")
        out = []
        for r in self._buf[:n]:
            out.append({k: getattr(r, k) for k, _ in dvc_result._fields_})
        return out

    def dvc_server_stats(self):
        a = (ctypes.c_int64 * 5)()
        self.ctx._rc(lib().dvc_server_stats(self.h, a), "dvc_server_stats")
        return dict(queued=a[0], resident=a[1], completed=a[2], rollout_slots=a[3], value_slots=a[4])

    def dvc_server_lanes(self):
        """Per lane: dict(context, players, tiles, mode, slots, resident, steps, step_us)."""
        a = (ctypes.c_int32 * (8 * 64))()
        n = lib().dvc_server_lanes(self.h, 64, a)
        if n < 0:
            self.ctx._rc(n, "dvc_server_lanes")
        keys = ("context", "players", "tiles", "mode", "slots", "resident", "steps", "step_us")
        return [dict(zip(keys, a[8 * i:8 * i + 8])) for i in range(min(n, 64))]

