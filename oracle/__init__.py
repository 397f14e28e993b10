"""CPU oracle for the Da Vinci Code MCTS of arXiv 2403.10720 (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  The plain single-threaded C statement of the method
lives in dvc_oracle.c; this module only loads it and marshals arguments.  Only
tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import it.

States cross this wrapper as 32-byte records in the boundary format (see the
comment above pack() in dvc_oracle.c), as numpy uint8 arrays of shape (n, 32).

Pin status per function:
  philox4x32_10 ..... pinned (published known-answer vectors)
  lnf ............... pinned (single precision, within 1 ulp of libm)
  init_states ....... pinned (rule invariants, deal sizes, history bounds)
  legal_count ....... pinned (88 root guesses of Sec. III-A, closed form I7)
  rollout / trace ... pinned (invariants, closed-form 1/k endgame, exact
                      win probabilities of tiny endgames by enumeration,
                      under both playout policies)
  det_count ......... pinned (brute-force enumeration of consistent deals)
  determinize ....... pinned (chi-square against uniform over those deals)
  mcts .............. pinned (UCB1 forced-win toy sequence, count invariants;
                      whole node tables of hand-solved 2- and 3-player
                      endgames, which fix the seat each node credits at
                      depths 1 to 3)
  mcts, value mode .. pinned (the same hand-solved endgames with a network
                      whose hidden weights are zero: each fresh leaf credits
                      round(p * playouts) per seat, p = softmax of the output
                      bias over the seats in play, relative to the mover)
  legal_actions ..... pinned (88 root guesses, canonical order written out;
                      ordering-aware policy: hand-made rows written out)
  play_move ......... pinned (hand-made positions: correct and wrong guesses,
                      elimination, empty pool, the draw that follows; STOP and
                      a kept turn in the full game of Fig. 2a)
  mcts, vanilla ..... pinned (plausible-set nodes against the determinizer's
                      samples: count, creation order, visits, the observer's
                      wins; joker places separate sets; a new set is a leaf;
                      the decision summed over sets)
  mcts, full tree ... pinned (a correct in-tree guess keeps the turn: STOP nodes
                      below it; visit-count invariants; the playout coin at a
                      may-stop leaf against exact enumeration)
  value_features .... pinned (hand-made positions with features written out)
  value_forward ..... pinned (closed form with zero hidden weights)
  value_loss_grad ... pinned (central finite differences in double)
  root_merge ........ pinned (one table reproduces or_mcts's own decision,
                      plain and vanilla; hand-made tables: sums that change
                      the winner, a tie to the lowest canonical rank)
  adamw_step ........ pinned (closed forms of the definition: the first step
                      from zero moments, a constant gradient over many steps,
                      weight decay on matrices only)
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


class _Cfg(ctypes.Structure):
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
class OracleConfig:
    nplayers: int = 2
    ntiles: int = 24
    deal: int = 4
    max_predraw: int = 0
    max_revealed: int = 5
    cont_thr: int = 1 << 31
    c_uct: float = 1.4142135623730951
    d_max: int = 8
    playouts: int = 1
    policy: int = 0
    tree_continue: int = 0
    vanilla: int = 0

    def c(self) -> _Cfg:
        return _Cfg(self.nplayers, self.ntiles, self.deal, self.max_predraw, self.max_revealed,
                    self.cont_thr, self.c_uct, self.d_max, self.playouts, self.policy, self.tree_continue,
                    self.vanilla)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        cfgp = ctypes.POINTER(_Cfg)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_philox4x32_10.restype = None
        L.or_lnf.argtypes = [ctypes.c_float]
        L.or_lnf.restype = ctypes.c_float
        L.or_init_states.argtypes = [cfgp, ctypes.c_uint64, ctypes.c_int, u8p]
        L.or_init_states.restype = ctypes.c_int
        L.or_legal_count.argtypes = [u8p]
        L.or_legal_count.restype = ctypes.c_int
        L.or_det_count.argtypes = [u8p, ctypes.c_int]
        L.or_det_count.restype = ctypes.c_uint64
        L.or_determinize.argtypes = [cfgp, u8p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_uint32, u8p]
        L.or_determinize.restype = ctypes.c_int
        L.or_rollout.argtypes = [cfgp, u8p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                 i32p, i64p]
        L.or_rollout.restype = ctypes.c_int
        L.or_playout_trace.argtypes = [cfgp, u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, u8p, ctypes.c_int]
        L.or_playout_trace.restype = ctypes.c_int
        L.or_play_move.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_uint32, u8p]
        L.or_play_move.restype = ctypes.c_int
        L.or_legal_actions.argtypes = [u8p, ctypes.c_int, i32p]
        L.or_legal_actions.restype = ctypes.c_int
        L.or_mcts.argtypes = [cfgp, u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, i32p,
                              ctypes.POINTER(ctypes.c_int), i32p]
        L.or_mcts.restype = ctypes.c_int
        L.or_mcts_value.argtypes = [cfgp, u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_float), i32p, ctypes.POINTER(ctypes.c_int), i32p]
        L.or_mcts_value.restype = ctypes.c_int
        L.or_mcts_work.argtypes = [cfgp, u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, i64p]
        L.or_mcts_work.restype = ctypes.c_int
        f32p = ctypes.POINTER(ctypes.c_float)
        f64p = ctypes.POINTER(ctypes.c_double)
        L.or_value_nparams.argtypes = []
        L.or_value_nparams.restype = ctypes.c_int
        L.or_value_features.argtypes = [u8p, f32p]
        L.or_value_features.restype = ctypes.c_int
        L.or_value_forward.argtypes = [f32p, u8p, f64p]
        L.or_value_forward.restype = ctypes.c_int
        L.or_value_loss_grad.argtypes = [f32p, u8p, f32p, ctypes.c_int, f64p]
        L.or_value_loss_grad.restype = ctypes.c_double
        L.or_adamw_step.argtypes = [f64p, f64p, f64p, f64p, ctypes.c_longlong, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_adamw_step.restype = ctypes.c_int
        L.or_root_merge.argtypes = [u8p, ctypes.c_int, i32p, i32p, ctypes.c_int, i32p]
        L.or_root_merge.restype = ctypes.c_int
        _lib = L
    return _lib


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _i32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _state(s):
    s = np.ascontiguousarray(np.asarray(s, dtype=np.uint8).reshape(32))
    return s


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def lnf(x: float) -> float:
    """The UCT logarithm, in IEEE single precision (argument rounded to float)."""
    return lib().or_lnf(float(x))


def init_states(cfg: OracleConfig, seed: int, n: int) -> np.ndarray:
    out = np.zeros((n, 32), dtype=np.uint8)
    c = cfg.c()
    rc = lib().or_init_states(ctypes.byref(c), seed, n, _u8(out))
    if rc:
        raise ValueError(f"or_init_states rc={rc}")
    return out


def legal_count(state) -> int:
    s = _state(state)
    return lib().or_legal_count(_u8(s))


def legal_actions(state, policy: int = 0) -> np.ndarray:
    """Legal guesses in canonical order as action codes (seat << 10 | slot << 5 | identity);
    policy 1: only those the ordering-aware playout policy keeps."""
    s = _state(state)
    out = np.zeros(3 * 26 * 26, dtype=np.int32)
    n = lib().or_legal_actions(_u8(s), int(policy), _i32(out))
    return out[:n].copy()


STOP = 0xFFF  # end a turn after a correct guess (full game tree, Fig. 2a)
SET = 0xFFE   # a plausible-number-set node of vanilla MCTS-dvc (Sec. III-A)


def play_move(state, code: int, seed: int, game: int, turn: int, cont: int = 0):
    """Returns (rc, next state): rc 0 played, 1 game already over, -1 illegal
    action.  cont = 1: a correct guess keeps the turn (the player may STOP)."""
    s = _state(state)
    out = np.zeros(32, dtype=np.uint8)
    rc = lib().or_play_move(_u8(s), int(code), int(cont), seed, game, turn, _u8(out))
    return rc, out


def det_count(state, observer: int = -1) -> int:
    s = _state(state)
    return int(lib().or_det_count(_u8(s), observer))


def determinize(cfg: OracleConfig, state, observer: int, seed: int, tree: int, it: int) -> np.ndarray:
    s = _state(state)
    out = np.zeros(32, dtype=np.uint8)
    c = cfg.c()
    rc = lib().or_determinize(ctypes.byref(c), _u8(s), observer, seed, tree, it, _u8(out))
    if rc:
        raise ValueError(f"or_determinize rc={rc}")
    return out


def rollout(cfg: OracleConfig, leaf, playouts: int, seed: int, tree: int, leaf_id: int):
    """Returns (wins per player (4,), RNG words consumed)."""
    s = _state(leaf)
    wins = np.zeros(4, dtype=np.int32)
    words = ctypes.c_int64(0)
    c = cfg.c()
    rc = lib().or_rollout(ctypes.byref(c), _u8(s), playouts, seed, tree, leaf_id, _i32(wins), ctypes.byref(words))
    if rc:
        raise ValueError(f"or_rollout rc={rc}")
    return wins, int(words.value)


def playout_trace(cfg: OracleConfig, leaf, seed: int, tree: int, j: int, leaf_id: int, maxlen: int = 256):
    s = _state(leaf)
    out = np.zeros((maxlen, 32), dtype=np.uint8)
    c = cfg.c()
    n = lib().or_playout_trace(ctypes.byref(c), _u8(s), seed, tree, j, leaf_id, _u8(out), maxlen)
    return out[:n]


VALUE_FEATURES = 640
VALUE_HIDDEN = 512


def value_nparams() -> int:
    return lib().or_value_nparams()


def value_features(state) -> np.ndarray:
    s = _state(state)
    out = np.zeros(VALUE_FEATURES, dtype=np.float32)
    lib().or_value_features(_u8(s), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return out


def value_forward(params, state) -> np.ndarray:
    """Win probability per absolute seat, computed in double."""
    prm = np.ascontiguousarray(params, dtype=np.float32)
    s = _state(state)
    out = np.zeros(4, dtype=np.float64)
    rc = lib().or_value_forward(prm.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _u8(s),
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc:
        raise ValueError("or_value_forward")
    return out


def value_loss_grad(params, states, labels):
    """(mean cross-entropy, gradient per parameter) in double."""
    prm = np.ascontiguousarray(params, dtype=np.float32)
    st = np.ascontiguousarray(np.asarray(states, dtype=np.uint8).reshape(-1, 32))
    lab = np.ascontiguousarray(np.asarray(labels, dtype=np.float32).reshape(-1, 4))
    g = np.zeros(value_nparams(), dtype=np.float64)
    loss = lib().or_value_loss_grad(prm.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _u8(st),
                                    lab.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(st),
                                    g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return loss, g


def mcts(cfg: OracleConfig, root, seed: int, tree: int, budget: int, value_params=None):
    """Returns (nodes (n, 4) int32 [action, parent, visits, wins] in creation
    order, best (4,) int32 [action, visits, wins, root visits]).  With
    value_params (the network's parameters, value_nparams() floats) the search
    runs in value mode: a fresh leaf that did not end in the tree credits each
    seat round(p * playouts) from the network instead of playing out."""
    s = _state(root)
    nodes = np.zeros((budget + 1, 4), dtype=np.int32)
    n = ctypes.c_int(0)
    best = np.zeros(4, dtype=np.int32)
    c = cfg.c()
    if value_params is None:
        rc = lib().or_mcts(ctypes.byref(c), _u8(s), seed, tree, budget, _i32(nodes), ctypes.byref(n), _i32(best))
    else:
        prm = np.ascontiguousarray(value_params, dtype=np.float32)
        assert prm.size == value_nparams()
        rc = lib().or_mcts_value(ctypes.byref(c), _u8(s), seed, tree, budget,
                                 prm.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _i32(nodes),
                                 ctypes.byref(n), _i32(best))
    if rc:
        raise ValueError(f"or_mcts rc={rc}")
    return nodes[: n.value].copy(), best


ADAMW = dict(b1=0.9, b2=0.999, eps=1e-8, wd=1e-4)


def adamw_step(w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step in double on copies of (w, m, v) with gradient g; t is
    the step number after the update.  Returns (w, m, v)."""
    n = value_nparams()
    arrs = [np.array(a, dtype=np.float64).reshape(n).copy() for a in (w, m, v)]
    gg = np.ascontiguousarray(np.asarray(g, dtype=np.float64).reshape(n))
    p = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs + [gg]]
    rc = lib().or_adamw_step(p[0], p[1], p[2], p[3], int(t), lr, b1, b2, eps, wd)
    if rc:
        raise ValueError("or_adamw_step")
    return tuple(arrs)


def mcts_work(cfg: OracleConfig, root, seed: int, tree: int, budget: int):
    """(random words, game steps) consumed by the playouts of or_mcts's search:
    one game step per guess, plus one per continue coin a playout from a
    may-stop leaf draws first."""
    s = _state(root)
    out = np.zeros(2, dtype=np.int64)
    c = cfg.c()
    rc = lib().or_mcts_work(ctypes.byref(c), _u8(s), seed, tree, budget, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc:
        raise ValueError(f"or_mcts_work rc={rc}")
    return int(out[0]), int(out[1])


def root_merge(root, tables, vanilla: int = 0):
    """Root-parallel merge (Sec. III-B) of K node tables of searches of one
    root: [action, visits, wins, root visits] of the summed decision."""
    s = _state(root)
    counts = np.array([len(t) for t in tables], dtype=np.int32)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.int32).reshape(-1, 4) for t in tables]))
    out = np.zeros(4, dtype=np.int32)
    rc = lib().or_root_merge(_u8(s), len(tables), _i32(flat), _i32(counts), int(vanilla), _i32(out))
    if rc:
        raise ValueError("or_root_merge")
    return out
