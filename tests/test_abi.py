"""The C-ABI library loads and exports every entry point include/dvc.h
declares (no compute calls; runs without a GPU)."""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2403_10720_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    import paper_2403_10720_gb300 as dvc
    names = dvc.declared_symbols()
    for must in ["dvc_create", "dvc_destroy", "dvc_init_states", "dvc_determinize", "dvc_rollout_batch",
                 "dvc_forest_create", "dvc_mcts_step", "dvc_mcts_select", "dvc_mcts_expand", "dvc_mcts_backprop",
                 "dvc_root_stats", "dvc_tree_export", "dvc_last_error", "dvc_check"]:
        assert must in names


def test_library_exports_every_declared_symbol(built):
    import paper_2403_10720_gb300 as dvc
    L = ctypes.CDLL(built)
    missing = [n for n in dvc.declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(built):
    import paper_2403_10720_gb300 as dvc
    L = dvc.lib()
    for n in dvc.declared_symbols():
        assert getattr(L, n).argtypes is not None or n in ("dvc_last_error",), n


def test_null_arguments_rejected_without_touching_the_device(built):
    import paper_2403_10720_gb300 as dvc
    L = dvc.lib()
    assert L.dvc_create(None, None, 0) == -1
    assert L.dvc_mcts_step(None, 1, 0, None) == -1
    assert L.dvc_rollout_batch(None, None, 0, 1, 0, None, None, None, None, None) == -1
    assert L.dvc_last_error(None) == b"null context"


def test_state_record_is_32_bytes():
    text = open(os.path.join(ROOT, "include", "dvc.h")).read()
    body = text[text.index("typedef struct dvc_state {"):text.index("} dvc_state;")]
    sizes = {"uint32_t": 4, "uint8_t": 1}
    total = 0
    for line in body.splitlines()[1:]:
        line = line.split("/*")[0].strip().rstrip(";")
        if not line:
            continue
        ty, name = line.split()
        n = int(name[name.index("[") + 1:name.index("]")]) if "[" in name else 1
        total += sizes[ty] * n
    assert total == 32
