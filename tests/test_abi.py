"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that the headers under include/ declare (no GPU needed: no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mvsk_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_25378_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("mvsk_create", "mvsk_set_prefs", "mvsk_solve", "mvsk_eval", "mvsk_solve_batch",
                 "mvsk_oracle_hvp", "mvsk_oracle_third", "mvsk_oracle_gram", "mvsk_oracle_ls",
                 "mvsk_destroy", "mvsk_last_error", "mvsk_column_stats", "mvsk_mlp_create", "mvsk_mlp_forward",
                 "mvsk_mlp_train_step", "mvsk_mlp_access", "mvsk_mlp_features", "mvsk_mlp_warm_start",
                 "mvsk_mlp_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert missing == []


def test_binding_loads_and_fails_loudly_without_library(tmp_path):
    import paper_2604_25378_gb300 as m
    with pytest.raises(ImportError):
        m._lib = None
        m.load(str(tmp_path / "missing.so"))
    m._lib = None
    assert m.load() is not None
