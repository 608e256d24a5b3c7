"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/bm.h declares (no compute calls: those need a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_29977_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("bm_analyze", "bm_factor", "bm_solve", "bm_query", "bm_destroy", "bm_workspace_bytes"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_the_same_symbols():
    from paper_2609_29977_gb300 import bm
    assert sorted(bm.EXPORTED_SYMBOLS) == declared_functions()


def test_host_only_entry_points(lib):
    from paper_2609_29977_gb300 import bm
    assert bm.bm_version() == 1
    assert "positive definite" in bm.bm_status_string(2)
    d = bm.make_desc(64, 64, 12, 4)
    n = bm.bm_workspace_bytes(d)
    # factors (3 blocks per stage) + level workspace (2) + vectors
    assert n >= 5 * 64 * 64 * 144 * 8
    assert bm.bm_workspace_bytes(bm.make_desc(0, 4, 4, 2)) == 0
    assert bm.bm_workspace_bytes(bm.make_desc(2, 4, 65, 2)) == 0
