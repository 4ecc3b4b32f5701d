"""Parity of the CUDA path (through the C ABI) with the CPU oracle, under the
mean-field gain rule (the departure kept as an option; the paper's gain has
its own file, tests/test_gpu_literal.py).  The preprocessing checks do not
depend on the rule; the run checks cover the mean-field kernels: the
persistent queue loop and its bounded barrier, the FP32 screen, the team,
block and hub tiers.

Integer and index results must be bit-exact: CSR, labels, orientation,
t(x,V), vt(x,V), node order, initial clustering, per-queue and per-iteration
memberships and community aggregates, community output.  Floating point:
the global cc and every WCC-hat(P) total are compared bit for bit (both sides
round the same expressions operation by operation and use correctly rounded
sums); the stated contract is 1e-9 relative, asserted as well.
"""
import math

import numpy as np
import pytest

from paper_2210_03211_gb300 import workloads as W

pytestmark = pytest.mark.gpu

T_REL = 1e-9


class _MeanField:
    """The binding (or the oracle) with every graph on the mean-field rule."""

    def __init__(self, mod):
        self._m = mod

    def __getattr__(self, k):
        return getattr(self._m, k)

    def Graph(self, *a, **kw):
        kw.setdefault("gain_rule", "meanfield")
        return self._m.Graph(*a, **kw)

    def OracleGraph(self, *a, **kw):
        g = self._m.OracleGraph(*a, **kw)
        g.set_gain_rule("meanfield")
        return g


@pytest.fixture(scope="module")
def lf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_03211_gb300 import build
    build.build()
    from paper_2210_03211_gb300 import lazyfox
    lazyfox.load_library()
    return _MeanField(lazyfox)


@pytest.fixture(scope="module")
def oracle_lib():
    import oracle
    oracle.build()
    return _MeanField(oracle)


def small_cases():
    cases = [W.from_pairs(W.clique(5) + W.clique(4, 10) + [(3, 10)], "two_cliques"),
             W.from_pairs([(0, 1), (0, 2), (1, 2), (2, 3), (2, 4), (3, 4)], "bowtie"),
             W.from_pairs(W.clique(4) + [(0, 4)], "k4_pendant"),
             W.from_pairs(W.path(5), "path5"),
             W.from_pairs(W.star(40), "star40"),
             W.from_pairs(W.cycle(3) + W.cycle(7, 10), "cycles")]
    for seed in range(4):
        cases.append(W.random_graph(n=60 + 20 * seed, m=400 + 100 * seed, seed=seed, self_loops=5, duplicates=20))
    cases.append(W.random_graph(n=300, m=1500, seed=11, hubs=3, hub_degree=250))
    cases.append(W.random_graph(n=3000, m=9000, seed=12, hubs=2, hub_degree=2600))
    cases.append(W.eu_core_like())
    cases.append(W.dblp_like(seed=3, scale=0.03))
    return cases


CASES = small_cases()
IDS = [c.name for c in CASES]


def compare_preprocessing(g, og):
    off, adj, labels = g.csr()
    ooff, oadj, olabels = og.csr()
    assert np.array_equal(labels, olabels)
    assert np.array_equal(off, ooff)
    assert np.array_equal(adj, oadj)
    # orientation: N+(u) = neighbours with higher (degree, id), ascending ids
    deg = np.diff(off)
    uoff, uadj = g.oriented()
    assert uoff[-1] == og.m
    for u in range(0, g.n, max(1, g.n // 500)):
        row = adj[off[u]:off[u + 1]]
        keep = row[(deg[row] > deg[u]) | ((deg[row] == deg[u]) & (row > u))]
        assert np.array_equal(uadj[uoff[u]:uoff[u + 1]], keep)
    t, vt, cc = g.node_stats()
    ot, ovt, occ = og.node_stats()
    assert np.array_equal(t, ot)
    assert np.array_equal(vt, ovt)
    assert cc == occ
    assert np.array_equal(g.order(), og.order())


def compare_state(g, og):
    s, o = g.state(), og.state()
    assert np.array_equal(s["mem_off"], o["mem_off"])
    assert np.array_equal(s["mem_ids"], o["mem_ids"])
    assert np.array_equal(s["n"], o["n"])
    assert np.array_equal(s["m"], o["m"])
    assert np.array_equal(s["vol"], o["vol"])


def compare_run(st, ref):
    assert st.iterations == ref["iterations"]
    assert st.converged == ref["converged"]
    assert st.wcc_initial == ref["T0"]
    assert np.array_equal(st.joins, ref["joins"])
    assert np.array_equal(st.leaves, ref["leaves"])
    for a, b in zip(st.wcc_history, ref["T"]):
        assert a == pytest.approx(b, rel=T_REL, abs=0)
        assert a == b


@pytest.mark.parametrize("el", CASES, ids=IDS)
def test_preprocessing_parity(lf, oracle_lib, el):
    og = oracle_lib.OracleGraph(el.src, el.dst)
    with lf.Graph(el.src, el.dst) as g:
        assert (g.n, g.m) == (og.n, og.m)
        compare_preprocessing(g, og)


@pytest.mark.parametrize("el", CASES, ids=IDS)
@pytest.mark.parametrize("q", [1, 2, 64, 1024, 1 << 30])
def test_run_parity(lf, oracle_lib, el, q):
    if q == 1 and el.num_edges > 20000:
        pytest.skip("queue size 1 is exercised on the smaller graphs")
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(q, 0.01, 50)
    with lf.Graph(el.src, el.dst) as g:
        st = g.run(q, 0.01, 50)
        compare_run(st, ref)
        compare_state(g, og)
        got = [c.tolist() for c in g.community_list()]
        want = [c.tolist() for c in og.communities()]
        assert got == want


@pytest.mark.parametrize("el", [CASES[-2], CASES[-4], CASES[-5]], ids=[IDS[-2], IDS[-4], IDS[-5]])
@pytest.mark.parametrize("q", [1, 7, 64])
def test_per_queue_parity(lf, oracle_lib, el, q):
    """State after an arbitrary number of queues, iteration ends included."""
    og = oracle_lib.OracleGraph(el.src, el.dst)
    nb = -(-og.n // q)
    points = sorted({1, 2, 3, nb - 1, nb, nb + 1, 2 * nb + 5} - {0})
    with lf.Graph(el.src, el.dst) as g:
        for b in points:
            og.run(q, -math.inf, 3, max_batches=b)
            g.run(q, -math.inf, 3, max_batches=b)
            compare_state(g, og)


@pytest.mark.parametrize("el", [CASES[-2], CASES[-4], CASES[-5], CASES[0]], ids=[IDS[-2], IDS[-4], IDS[-5], IDS[0]])
def test_block_tier_and_row_growth(lf, oracle_lib, el):
    """Force every node onto the block-wide evaluation path and start from a
    membership capacity of 2 so that the rows must grow."""
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(16, -math.inf, 6)
    with lf.Graph(el.src, el.dst, warp_max_degree=1, member_slots=2) as g:
        st = g.run(16, -math.inf, 6)
        compare_run(st, ref)
        compare_state(g, og)


def test_graph_replay_equals_direct_launches_and_reruns(lf, oracle_lib):
    el = W.eu_core_like(seed=2)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(32, 0.01, 50)
    with lf.Graph(el.src, el.dst, per_queue_launches=True, use_graphs=False) as g1, \
            lf.Graph(el.src, el.dst, per_queue_launches=True) as g2:
        a = g1.run(32, 0.01, 50)
        b = g2.run(32, 0.01, 50)
        c = g2.run(32, 0.01, 50)    # same handle again: restarts from the initial clustering
        for st in (a, b, c):
            compare_run(st, ref)
        compare_state(g2, og)


def test_device_edge_input_equals_host_input(lf, oracle_lib):
    import torch
    el = W.eu_core_like(seed=4)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(8, 0.01, 50)
    s = torch.from_numpy(el.src).cuda()
    d = torch.from_numpy(el.dst).cuda()
    with lf.Graph(s, d) as g:
        compare_preprocessing(g, og)
        compare_run(g.run(8, 0.01, 50), ref)
    with lf.Graph(el.src, el.dst, allocator="cuda") as g:
        compare_run(g.run(8, 0.01, 50), ref)


def test_edge_cases(lf, oracle_lib):
    # empty edge list
    with lf.Graph(np.zeros(0, np.int32), np.zeros(0, np.int32)) as g:
        assert (g.n, g.m) == (0, 0)
        st = g.run(4, 0.01, 5)
        assert st.iterations == 1 and st.wcc_initial == 0.0
        off, mem = g.communities()
        assert off.tolist() == [0] and mem.shape[0] == 0
    # only self-loops and duplicates of one edge; ids near the int32 limit
    big = 2**31 - 1
    src = np.array([5, 5, big, big - 7, big], np.int32)
    dst = np.array([5, 5, big - 7, big, big - 7], np.int32)
    og = oracle_lib.OracleGraph(src, dst)
    with lf.Graph(src, dst) as g:
        assert (g.n, g.m) == (2, 1)
        compare_preprocessing(g, og)
        compare_run(g.run(1, 0.01, 10), og.run(1, 0.01, 10))
    # max_iters = 0: the initial clustering is the result (singletons kept)
    el = W.from_pairs(W.clique(4) + [(0, 4)])
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(1, 0.01, 0)
    with lf.Graph(el.src, el.dst) as g:
        st = g.run(1, 0.01, 0)
        assert st.iterations == 0 and st.wcc_initial == ref["T0"]
        assert [c.tolist() for c in g.community_list()] == [[0, 1, 2, 3], [4]]
    # invalid arguments
    with pytest.raises(lf.LazyFoxError):
        lf.Graph(np.array([0, -3], np.int32), np.array([1, 2], np.int32))
    with lf.Graph(el.src, el.dst) as g:
        with pytest.raises(lf.LazyFoxError):
            g.run(0, 0.01, 5)
        with pytest.raises(lf.LazyFoxError):
            g.run(4, 0.01, -1)
        with pytest.raises(lf.LazyFoxError):
            g.communities()   # before any run


@pytest.mark.parametrize("q", [64, 1024])
def test_full_size_335k_parity(lf, oracle_lib, q):
    """The 335k-node / ~0.93M-edge workload at full size, in the configuration
    the benchmark times: every output compared with the oracle, with the
    default launch shape and with the shape the autotuner picks for the
    benchmark (two-iteration trials)."""
    el = W.dblp_like()
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(q, 0.01, 50)
    want = og.communities()
    with lf.Graph(el.src, el.dst) as g:
        compare_preprocessing(g, og)
        for tuned in (False, True):
            if tuned:
                g.autotune(q, 2)
            st = g.run(q, 0.01, 50)
            compare_run(st, ref)
            compare_state(g, og)
            off, mem = g.communities()
            assert off.shape[0] - 1 == len(want)
            assert np.array_equal(mem, np.concatenate(want))


@pytest.mark.parametrize("el", [CASES[-1], CASES[-2], CASES[-4]], ids=[IDS[-1], IDS[-2], IDS[-4]])
def test_fp32_screen_changes_no_decision(lf, oracle_lib, el):
    """The FP32 screen only rules out candidates that cannot be the best
    action: evaluating every candidate in FP64 gives the same run."""
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(64, -math.inf, 5)
    with lf.Graph(el.src, el.dst, exhaustive_fp64=True) as g1, lf.Graph(el.src, el.dst) as g2:
        a = g1.run(64, -math.inf, 5)
        b = g2.run(64, -math.inf, 5)
        compare_run(a, ref)
        compare_run(b, ref)
        s1, s2 = g1.state(), g2.state()
        for k in s1:
            assert np.array_equal(s1[k], s2[k])


@pytest.mark.parametrize("el", [CASES[-1], CASES[-2], CASES[-4], CASES[1]], ids=[IDS[-1], IDS[-2], IDS[-4], IDS[1]])
@pytest.mark.parametrize("q", [1, 64, 4096])
def test_persistent_loop_equals_per_queue_launches(lf, oracle_lib, el, q):
    """The persistent queue kernel and two launches per queue give
    the oracle's run, queue for queue."""
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(q, 0.01, 50)
    with lf.Graph(el.src, el.dst, per_queue_launches=True) as g1, lf.Graph(el.src, el.dst, per_queue_launches=False) as g2:
        compare_run(g1.run(q, 0.01, 50), ref)
        compare_run(g2.run(q, 0.01, 50), ref)
        compare_state(g2, og)


def test_barrier_timeout_is_reported_and_recoverable(lf, oracle_lib):
    """A block that never reaches the grid barrier (injected on the host side
    of the test through an option) makes every bounded wait run out: the call
    returns LF_ERR_TIMEOUT instead of hanging, and the GPU stays usable."""
    el = W.eu_core_like(seed=6)
    with lf.Graph(el.src, el.dst, inject_barrier_stall=True, barrier_timeout_ms=50, per_queue_launches=False) as g:
        with pytest.raises(lf.LazyFoxError) as ei:
            g.run(64, 0.01, 5)
        assert ei.value.status == lf.LF_ERR_TIMEOUT
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(64, 0.01, 50)
    with lf.Graph(el.src, el.dst) as g:
        compare_run(g.run(64, 0.01, 50), ref)


@pytest.mark.parametrize("el", [CASES[-1], CASES[-2], CASES[-4], CASES[-5]], ids=[IDS[-1], IDS[-2], IDS[-4], IDS[-5]])
@pytest.mark.parametrize("team", [1, 2, 4, 8])
@pytest.mark.parametrize("per_queue", [False, True])
def test_team_sizes_give_the_same_run(lf, oracle_lib, el, team, per_queue):
    """1, 2, 4 or 8 warps per evaluated node, persistent or per-queue launches:
    the same actions as the oracle, queue for queue."""
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(48, -math.inf, 4)
    with lf.Graph(el.src, el.dst, warps_per_node=team, per_queue_launches=per_queue) as g:
        compare_run(g.run(48, -math.inf, 4), ref)
        compare_state(g, og)


@pytest.mark.parametrize("spokes,leaves,leaf_degree", [(2100, 20000, 252), (600, 5000, 140)])
def test_triangle_tiers_parity(lf, oracle_lib, spokes, leaves, leaf_degree):
    """Out-degrees beyond one warp's list (129-2048: the block walk; above
    2048: the big-node kernel) next to short ones: t(x,V), vt(x,V), order and
    cc bit-exact, then two iterations with every node hub-sized."""
    el = W.wide_fan(spokes, leaves, leaf_degree, chords=5000, seed=spokes)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(4096, -math.inf, 2)
    with lf.Graph(el.src, el.dst) as g:
        compare_preprocessing(g, og)
        compare_run(g.run(4096, -math.inf, 2), ref)
        compare_state(g, og)


@pytest.mark.parametrize("q", [4096, 1 << 30])
def test_hub_with_many_candidates(lf, oracle_lib, q):
    """A hub whose neighbours bring over 10,000 distinct communities: its
    candidates are screened and evaluated by several blocks.  Every output
    equal to the oracle's."""
    el = W.hub_of_triangles(12000, extra=2, seed=3)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(q, -math.inf, 3)
    with lf.Graph(el.src, el.dst) as g:
        compare_preprocessing(g, og)
        compare_run(g.run(q, -math.inf, 3), ref)
        compare_state(g, og)


@pytest.mark.parametrize("q", [1024, 65536])
def test_large_shape_scaled_parity(lf, oracle_lib, q):
    """The 3.07M-node workload's shape (Chung-Lu exponent 2.2, community sizes
    10-5,000, heavy hubs) at 2% scale, at the large queue sizes, 20 iterations
    without early stop: every output equal to the oracle's."""
    el = W.large_like(scale=0.02)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(q, -math.inf, 20)
    with lf.Graph(el.src, el.dst) as g:
        compare_preprocessing(g, og)
        compare_run(g.run(q, -math.inf, 20), ref)
        compare_state(g, og)


def _recount(off, adj, s):
    """n_C, m_C and vol_C recounted from memberships (numpy, any size)."""
    n = off.shape[0] - 1
    k = s["n"].shape[0]
    cnt = np.diff(s["mem_off"])
    node_of = np.repeat(np.arange(n), cnt)
    deg = np.diff(off)
    n_c = np.bincount(s["mem_ids"], minlength=k)
    vol_c = np.bincount(s["mem_ids"], weights=deg[node_of], minlength=k).astype(np.int64)
    # internal edges: pairs (x, y) adjacent with a common community, counted per community
    key = node_of.astype(np.int64) * (k + 1) + s["mem_ids"]
    order = np.argsort(key)
    key = key[order]
    src = np.repeat(np.arange(n), deg)
    m2 = np.zeros(k, np.int64)
    for lo in range(0, n, 200_000):   # node blocks keep memory bounded
        hi = min(n, lo + 200_000)
        e0, e1 = off[lo], off[hi]
        xs, ys = src[e0:e1], adj[e0:e1]
        a0, a1 = s["mem_off"][xs], s["mem_off"][xs + 1]
        reps = a1 - a0
        xi = np.repeat(np.arange(xs.shape[0]), reps)
        cs = s["mem_ids"][np.repeat(a0, reps) + (np.arange(reps.sum()) - np.repeat(np.cumsum(reps) - reps, reps))]
        q = ys[xi].astype(np.int64) * (k + 1) + cs
        hit = np.searchsorted(key, q)
        ok = (hit < key.shape[0]) & (key[np.minimum(hit, key.shape[0] - 1)] == q)
        m2 += np.bincount(cs[ok], minlength=k)
    return n_c, m2 // 2, vol_c


@pytest.mark.skipif(not __import__("os").environ.get("LF_TEST_LARGE"), reason="set LF_TEST_LARGE=1 (several minutes)")
def test_large_full_size_sampled(lf, oracle_lib):
    """Full 3.07M-node / ~115M-edge workload at queue size 65536: preprocessing
    equal to the oracle's (CSR and labels), t(x,V) and vt(x,V) on sampled
    nodes by the oracle's per-node count, the node order consistent with
    those counts, and after the run every community aggregate equal to its
    recount from the memberships."""
    el = W.large_like()
    og = oracle_lib.OracleGraph(el.src, el.dst, prepare=False)
    with lf.Graph(el.src, el.dst) as g:
        off, adj, labels = g.csr()
        ooff, oadj, olabels = og.csr()
        assert np.array_equal(labels, olabels) and np.array_equal(off, ooff) and np.array_equal(adj, oadj)
        t, vt, cc = g.node_stats()
        rng = np.random.default_rng(0)
        deg = np.diff(off)
        sample = np.concatenate([rng.choice(g.n, 150, replace=False), np.argsort(deg)[-50:]])
        for x in sample:
            assert (t[x], vt[x]) == og.node_triangles(int(x)), x
        order = g.order()
        for a in range(0, g.n - 1, 997):   # sampled neighbours in the order, compared exactly
            xa, xb = int(order[a]), int(order[a + 1])
            ca = (int(t[xa]), int(deg[xa]) * (int(deg[xa]) - 1) // 2) if deg[xa] > 1 else (0, 1)
            cb = (int(t[xb]), int(deg[xb]) * (int(deg[xb]) - 1) // 2) if deg[xb] > 1 else (0, 1)
            lhs, rhs = ca[0] * cb[1], cb[0] * ca[1]
            assert lhs > rhs or (lhs == rhs and (deg[xa] > deg[xb] or (deg[xa] == deg[xb] and xa < xb)))
        st = g.run(65536, -math.inf, 20)
        assert st.iterations == 20
        s = g.state()
        n_c, m_c, vol_c = _recount(off, adj, s)
        assert np.array_equal(n_c, s["n"]) and np.array_equal(m_c, s["m"]) and np.array_equal(vol_c, s["vol"])


@pytest.mark.parametrize("hub_degree,q", [(64, 1024), (64, 4096), (128, 65536)])
def test_hub_degree_threshold_gives_the_same_run(lf, oracle_lib, hub_degree, q):
    """Many more nodes on the hub path (global tables, second stream): the
    run is the oracle's, bit for bit."""
    el = W.large_like(scale=0.02)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(q, -math.inf, 5)
    with lf.Graph(el.src, el.dst, hub_degree=hub_degree) as g:
        compare_run(g.run(q, -math.inf, 5), ref)
        compare_state(g, og)
