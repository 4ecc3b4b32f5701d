"""The allocation-free triangle entry point (lf_triangles_noalloc), for
callers that cannot allocate device memory when they call it.

Called twice in a row through the C ABI on the same inputs; each time its
t(x,V) and vt(x,V) must equal what lf_graph_create computed (integers: exact).
This file is collected last so that a run stopping at the first failure has
run every other test before it; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2210_03211_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_03211_gb300 import build
    build.build()
    from paper_2210_03211_gb300 import lazyfox
    lazyfox.load_library()
    return lazyfox


@pytest.mark.parametrize("make", [lambda: W.dblp_like(seed=5, scale=0.05), lambda: W.wide_fan(seed=9)],
                         ids=["dblp_like_5pct", "wide_fan"])
def test_noalloc_triangles_equal_the_allocating_path_twice(lf, oracle_lib, make):
    import torch
    el = make()
    with lf.Graph(el.src, el.dst) as g:
        t_ref, vt_ref, _ = g.node_stats()
        ooff, oadj = g.oriented()
        n, m = g.n, g.m
    # the allocating path is itself the oracle's (triangles by sorted merges)
    ot, ovt, _ = oracle_lib.OracleGraph(el.src, el.dst).node_stats()
    assert np.array_equal(t_ref, ot) and np.array_equal(vt_ref, ovt)
    L = lf.load_library()
    d_ooff = torch.from_numpy(ooff).cuda()
    d_oadj = torch.from_numpy(oadj).cuda()
    d_t = torch.empty(n, dtype=torch.int64, device="cuda")
    d_vt = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        d_t.fill_(-7)      # stale values must not leak through
        d_vt.fill_(-7)
        st = L.lf_triangles_noalloc(C.c_void_p(d_ooff.data_ptr()), C.c_void_p(d_oadj.data_ptr()), n, m,
                                    C.c_void_p(d_t.data_ptr()), C.c_void_p(d_vt.data_ptr()),
                                    C.c_void_p(stream.cuda_stream))
        assert st == lf.LF_OK, L.lf_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(d_t.cpu().numpy(), t_ref), f"call {call}"
        assert np.array_equal(d_vt.cpu().numpy(), vt_ref), f"call {call}"
        assert np.array_equal(d_t.cpu().numpy(), ot) and np.array_equal(d_vt.cpu().numpy(), ovt), f"call {call}"


def test_noalloc_rejects_a_malformed_csr(lf):
    """Offsets that do not end at num_edges, or a neighbour id outside the
    nodes, are rejected (LF_ERR_INVALID) before any counting kernel runs."""
    import torch
    L = lf.load_library()
    n, m = 4, 3
    t = torch.zeros(n, dtype=torch.int64, device="cuda")
    vt = torch.zeros(n, dtype=torch.int32, device="cuda")
    good_off = torch.tensor([0, 2, 3, 3, 3], dtype=torch.int64, device="cuda")
    for off, adj in ((torch.tensor([0, 2, 3, 3, 5], dtype=torch.int64, device="cuda"),
                      torch.tensor([1, 2, 2], dtype=torch.int32, device="cuda")),
                     (good_off, torch.tensor([1, 2, 9], dtype=torch.int32, device="cuda")),
                     (torch.tensor([0, 3, 2, 3, 3], dtype=torch.int64, device="cuda"),
                      torch.tensor([1, 2, 2], dtype=torch.int32, device="cuda"))):
        st = L.lf_triangles_noalloc(C.c_void_p(off.data_ptr()), C.c_void_p(adj.data_ptr()), n, m,
                                    C.c_void_p(t.data_ptr()), C.c_void_p(vt.data_ptr()), None)
        assert st == lf.LF_ERR_INVALID, L.lf_last_error()
        assert b"malformed" in L.lf_last_error()
    # and a well-formed one still works afterwards (a triangle 0-1-2 and node 3 alone)
    adj = torch.tensor([1, 2, 2], dtype=torch.int32, device="cuda")
    st = L.lf_triangles_noalloc(C.c_void_p(good_off.data_ptr()), C.c_void_p(adj.data_ptr()), n, m,
                                C.c_void_p(t.data_ptr()), C.c_void_p(vt.data_ptr()), None)
    assert st == lf.LF_OK, L.lf_last_error()
    torch.cuda.synchronize()
    assert t.cpu().tolist() == [1, 1, 1, 0] and vt.cpu().tolist() == [2, 2, 2, 0]


def test_noalloc_rejects_sizes_beyond_its_array(lf):
    L = lf.load_library()
    st = L.lf_triangles_noalloc(None, None, 1 << 20, 20 << 20, None, None, None)
    assert st == lf.LF_ERR_CAPACITY
    assert b"16 MiB" in L.lf_last_error()
