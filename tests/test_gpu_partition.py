"""Inserted divisions and per-iteration results on the GPU (through the C
ABI), against the oracle: a division replaces the initial clustering
(Methods, Initial Clustering), and the communities saved after an iteration
continue the run exactly when inserted again."""
import math

import numpy as np
import pytest

from paper_2210_03211_gb300 import workloads as W
from test_gpu_parity import compare_run, compare_state

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


def _planted(el, og):
    _, _, labels = og.csr()
    comms = [np.unique(np.asarray(c, dtype=np.int32)) for c in el.planted]
    comms = [c[np.isin(c, labels)] for c in comms]
    return [c for c in comms if c.shape[0] > 0]


@pytest.mark.parametrize("q", [1, 16, 1 << 30])
def test_inserted_planted_cover(lf, oracle_lib, q):
    el = W.eu_core_like()
    og = oracle_lib.OracleGraph(el.src, el.dst)
    comms = _planted(el, og)
    og.set_partition(comms)
    ref = og.run(q, 0.01, 50)
    with lf.Graph(el.src, el.dst) as g:
        g.set_partition(comms)
        compare_run(g.run(q, 0.01, 50), ref)
        compare_state(g, og)


@pytest.mark.parametrize("q", [64, 4096])
def test_inserted_cover_power_law(lf, oracle_lib, q):
    el = W.dblp_like(seed=3, scale=0.03)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    comms = _planted(el, og)
    og.set_partition(comms)
    ref = og.run(q, -math.inf, 4)
    with lf.Graph(el.src, el.dst) as g:
        g.set_partition(comms)
        compare_run(g.run(q, -math.inf, 4), ref)
        compare_state(g, og)


@pytest.mark.parametrize("q,a,b", [(1, 2, 2), (256, 1, 3), (1 << 30, 3, 2)])
def test_resume_equals_one_run(lf, oracle_lib, q, a, b):
    el = W.random_graph(n=2000, m=12000, seed=21, hubs=2, hub_degree=700)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(q, -math.inf, a + b)
    with lf.Graph(el.src, el.dst) as g:
        first = g.run(q, -math.inf, a)
        g.set_partition(g.communities())
        second = g.run(q, -math.inf, b)
        assert second.wcc_initial == first.wcc_history[-1] == ref["T"][a - 1]
        assert np.array_equal(np.concatenate([first.wcc_history, second.wcc_history]), ref["T"])
        assert np.array_equal(np.concatenate([first.joins, second.joins]), ref["joins"])
        assert np.array_equal(np.concatenate([first.leaves, second.leaves]), ref["leaves"])
        got = [c.tolist() for c in g.community_list()]
        assert got == [c.tolist() for c in og.communities()]


def test_iteration_callback_sees_each_iterations_communities(lf, oracle_lib):
    el = W.eu_core_like()
    seen = {}
    with lf.Graph(el.src, el.dst) as g:
        def cb(it, wcc):
            seen[it] = (wcc, [c.tolist() for c in g.community_list()])
            return it == 3   # stop after the third iteration
        st = g.run(8, -math.inf, 10, on_iteration=cb)
        assert st.iterations == 3 and not st.converged
        assert sorted(seen) == [1, 2, 3]
    for k in (1, 2, 3):
        og = oracle_lib.OracleGraph(el.src, el.dst)
        ref = og.run(8, -math.inf, k)
        assert seen[k][0] == ref["T"][-1]
        assert seen[k][1] == [c.tolist() for c in og.communities()]


def test_invalid_divisions(lf):
    el = W.from_pairs(W.clique(4) + [(3, 10)], "k4_tail")
    with lf.Graph(el.src, el.dst) as g:
        for bad in ([np.array([0, 1, 99], np.int32)], [np.array([0, 1, 1], np.int32)]):
            with pytest.raises(lf.LazyFoxError) as e:
                g.set_partition(bad)
            assert e.value.status == lf.LF_ERR_INVALID
        with pytest.raises(lf.LazyFoxError) as e:
            g.set_partition([np.array([0], np.int32)] * 6)   # more communities than nodes
        assert e.value.status == lf.LF_ERR_CAPACITY
        with pytest.raises(lf.LazyFoxError) as e:
            g.set_partition((np.array([0, 2, 1], np.int64), np.array([0, 1], np.int32)))
        assert e.value.status == lf.LF_ERR_INVALID
        g.set_partition(None)
        assert g.run(1, 0.01, 5).iterations >= 1
