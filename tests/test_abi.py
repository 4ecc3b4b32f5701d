"""The C-ABI library builds, loads and exports every entry point that
include/lazyfox.h declares (no GPU needed; no compute call is made)."""
import ctypes as C
import os
import re

import numpy as np
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
    # lf_options: 4 pointers + 14 int32 = 88 bytes on LP64
    assert C.sizeof(lazyfox.Options) == 4 * 8 + 14 * 4
    assert C.sizeof(lazyfox.CreateStatsC) == 3 * 8 + 5 * 8 + 8 + 8
    assert C.sizeof(lazyfox.TuneResultC) == 4 * 4 + 2 * 8
    assert C.sizeof(lazyfox.ServerOptionsC) == 8 + 4 + 4
    assert C.sizeof(lazyfox.JobResultC) == 4 * 4 + 2 * 8 + 4 * 8 + 3 * 8
    assert C.sizeof(lazyfox.RunStatsC) == 4 + 4 + 8 + 8 + 8 + 8 + 8 + 8 + 8 + 8 + 3 * 8 + 4 * 8 + 4 * 8 + 2 * 8


def test_product_path_has_no_oracle_or_fallback():
    pkg = os.path.join(ROOT, "paper_2210_03211_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lazyfox_oracle" not in text, f


def test_binding_has_a_function_per_entry_point():
    from paper_2210_03211_gb300 import lazyfox
    missing = [f for f in declared_functions() if not callable(getattr(lazyfox, f, None))]
    assert missing == []


class _Recorder:
    """Stands in for a Graph / Batch / Server handle: records the method calls."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if name.startswith("_"):
            raise AttributeError(name)

        def method(*args, **kw):
            self.calls.append((name, args, kw))
            return name
        return method


def test_same_name_functions_reach_the_handle_methods():
    from paper_2210_03211_gb300 import lazyfox as L
    g = _Recorder()
    assert L.lf_run(g, 64, 0.01, 7) == "run" and g.calls[-1] == ("run", (64, 0.01, 7), {})
    assert L.lf_run_partial(g, 8, 0.5, 3, 11) == "run"
    assert g.calls[-1] == ("run", (8, 0.5, 3), {"max_batches": 11})
    for fn, meth in ((L.lf_get_communities, "communities"), (L.lf_get_node_stats, "node_stats"),
                     (L.lf_get_create_stats, "create_stats"), (L.lf_get_csr, "csr"),
                     (L.lf_get_oriented, "oriented"), (L.lf_get_order, "order"), (L.lf_get_state, "state"),
                     (L.lf_graph_destroy, "close"), (L.lf_batch_get_info, "info"),
                     (L.lf_batch_get_communities, "graph_communities"), (L.lf_server_destroy, "close")):
        fn(g)
        assert g.calls[-1][0] == meth, fn.__name__
    L.lf_set_partition(g, [[1, 2]])
    assert g.calls[-1] == ("set_partition", ([[1, 2]],), {})
    L.lf_batch_get_history(g, 3)
    assert g.calls[-1] == ("history", (3,), {})
    L.lf_autotune(g, 256, 2)
    assert g.calls[-1] == ("autotune", (256, 2), {})
    L.lf_server_submit(g, "s", "d", 16, 0.1, 4)
    assert g.calls[-1] == ("submit", ("s", "d", 16, 0.1, 4), {})
    L.lf_server_wait(g, 5, 1.5)
    assert g.calls[-1] == ("wait", (5, 1.5), {})
    L.lf_server_get_communities(g, 5)
    assert g.calls[-1] == ("community_list", (5,), {})
    L.lf_server_release(g, 5)
    assert g.calls[-1] == ("release", (5,), {})


def test_lf_get_sizes_and_lf_last_error(lib):
    from paper_2210_03211_gb300 import lazyfox as L

    class FakeLib:
        def lf_get_sizes(self, h, n, m):
            n._obj.value, m._obj.value = 12, 34
            return L.LF_OK

    g = _Recorder()
    g._L, g._h = FakeLib(), C.c_void_p(1)
    assert L.lf_get_sizes(g) == (12, 34)
    assert lib.lf_run(None, 4, 0.01, 3, None) == L.LF_ERR_INVALID
    assert "NULL" in L.lf_last_error()


def test_iteration_callback_set_by_name_reaches_the_run():
    """lf_set_iteration_callback stores the callback; Graph.run passes it to
    the library, which calls it after each iteration (a fake library here)."""
    from paper_2210_03211_gb300 import lazyfox as L

    class FakeLib:
        cb = None

        def lf_set_iteration_callback(self, h, cb, ctx):
            self.cb = cb if cb else None
            return L.LF_OK

        def lf_run(self, h, q, thr, iters, st):
            stats = st._obj
            for it in (1, 2):
                stats.wcc_history[it - 1] = 10.0 * it
                stats.iterations = it
                if self.cb is not None and self.cb(None, it, 10.0 * it, None):
                    break
            return L.LF_OK

    g = L.Graph.__new__(L.Graph)
    g._L, g._h = FakeLib(), C.c_void_p(1)
    seen = []
    L.lf_set_iteration_callback(g, lambda it, wcc: seen.append((it, wcc)) or it >= 1)
    st = L.lf_run(g, 4, 0.01, 5)
    assert seen == [(1, 10.0)] and st.iterations == 1
    assert g._L.cb is None   # removed after the run
    L.lf_set_iteration_callback(g, None)
    assert L.lf_run(g, 4, 0.01, 5).iterations == 2
    g._h = C.c_void_p()   # nothing to destroy


def test_same_name_entry_points_fail_loudly_without_a_gpu(lib):
    import torch
    from paper_2210_03211_gb300 import lazyfox as L
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.LazyFoxError) as e:
        L.lf_graph_create(np.array([0], np.int32), np.array([1], np.int32))
    assert e.value.status == L.LF_ERR_CUDA
    with pytest.raises(TypeError):
        L.lf_triangles_noalloc(torch.zeros(2, dtype=torch.int64), torch.zeros(1, dtype=torch.int32),
                               torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int32))
