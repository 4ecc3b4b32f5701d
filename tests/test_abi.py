"""The C-ABI library builds, loads and exports every entry point that
include/lazyfox.h declares (no GPU needed; no compute call is made)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lazyfox.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_03211_gb300 import build
    build.build()
    from paper_2210_03211_gb300 import lazyfox
    return lazyfox.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lf_graph_create", "lf_run", "lf_get_communities", "lf_get_node_stats",
                     "lf_graph_destroy", "lf_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert missing == []


def test_binding_covers_the_header(lib):
    from paper_2210_03211_gb300 import lazyfox
    assert sorted(lazyfox.ABI_FUNCTIONS) == declared_functions()


def test_null_handle_is_rejected_without_touching_the_gpu(lib):
    from paper_2210_03211_gb300 import lazyfox
    assert lib.lf_run(None, 4, 0.01, 3, None) == lazyfox.LF_ERR_INVALID
    assert b"NULL" in lib.lf_last_error()
    assert lib.lf_get_sizes(None, None, None) == lazyfox.LF_ERR_INVALID
    lib.lf_graph_destroy(None)


def test_struct_layouts_match_header():
    from paper_2210_03211_gb300 import lazyfox
    # lf_options: 4 pointers + 11 int32 (+4 padding) = 80 bytes on LP64
    assert C.sizeof(lazyfox.Options) == 4 * 8 + 12 * 4
    assert C.sizeof(lazyfox.CreateStatsC) == 3 * 8 + 5 * 8 + 8 + 8
    assert C.sizeof(lazyfox.TuneResultC) == 4 * 4 + 2 * 8
    assert C.sizeof(lazyfox.ServerOptionsC) == 8 + 4 + 4
    assert C.sizeof(lazyfox.JobResultC) == 4 * 4 + 2 * 8 + 4 * 8 + 3 * 8
    assert C.sizeof(lazyfox.RunStatsC) == 4 + 4 + 8 + 8 + 8 + 8 + 8 + 8 + 8 + 8 + 3 * 8 + 4 * 8 + 4 * 8


def test_product_path_has_no_oracle_or_fallback():
    pkg = os.path.join(ROOT, "paper_2210_03211_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lazyfox_oracle" not in text, f
