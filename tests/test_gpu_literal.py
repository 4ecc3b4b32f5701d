"""Parity of the CUDA path with the oracle under the paper's gain rule.

The gain of a move is the change of WCC-hat(P) (Node Changes: Joining /
Leaving a Community, with the WCC-hat sum equations): the moved community's
member terms after and before the move plus the node's own term, summed
exactly.  Both sides take every decision from the correctly rounded value of
that sum (the GPU brackets candidates first and evaluates the undecided ones
exactly), so memberships, joins, leaves and every WCC-hat(P) must be equal
bit for bit; the stated contract for the totals, 1e-9 relative, is asserted
too.  Through the C ABI on the GPU.
"""
import math

import numpy as np
import pytest

from paper_2210_03211_gb300 import workloads as W

pytestmark = pytest.mark.gpu

T_REL = 1e-9
RULE = "literal"


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


def cases():
    out = [W.from_pairs(W.clique(5) + W.clique(4, 10) + [(3, 10)], "two_cliques"),
           W.from_pairs([(0, 1), (0, 2), (1, 2), (2, 3), (2, 4), (3, 4)], "bowtie"),
           W.from_pairs([(0, 1), (0, 2), (1, 2), (2, 3), (3, 4)], "triangle_tail"),
           W.from_pairs(W.path(5), "path5"),
           W.from_pairs(W.star(40), "star40")]
    for seed in range(3):
        out.append(W.random_graph(n=60 + 20 * seed, m=400 + 100 * seed, seed=seed, self_loops=5, duplicates=20))
    out.append(W.planted_er(n=300, num_comms=10, seed=3))
    out.append(W.random_graph(n=300, m=1500, seed=11, hubs=3, hub_degree=250))
    out.append(W.random_graph(n=3000, m=9000, seed=12, hubs=2, hub_degree=2600))
    out.append(W.eu_core_like())
    out.append(W.dblp_like(seed=3, scale=0.03))
    return out


CASES = cases()
IDS = [c.name for c in CASES]


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


def check_run(lf, og, el, q, thr=0.01, iters=50, **kw):
    ref = og.run(q, thr, iters, rule=RULE)
    with lf.Graph(el.src, el.dst, gain_rule=RULE, **kw) as g:
        st = g.run(q, thr, iters)
        compare_run(st, ref)
        compare_state(g, og)
        assert [c.tolist() for c in g.community_list()] == [c.tolist() for c in og.communities()]
    return ref


@pytest.mark.parametrize("el", CASES, ids=IDS)
@pytest.mark.parametrize("q", [1, 2, 7, 64, 1024, 1 << 30])
def test_literal_run_parity(lf, oracle_lib, el, q):
    if q == 1 and el.num_edges > 20000:
        pytest.skip("queue size 1 is exercised on the smaller graphs")
    check_run(lf, oracle_lib.OracleGraph(el.src, el.dst), el, q)


@pytest.mark.parametrize("idx", [-1, -2, -5], ids=[IDS[-1], IDS[-2], IDS[-5]])
@pytest.mark.parametrize("q", [1, 7, 64])
def test_literal_per_queue_parity(lf, oracle_lib, idx, q):
    """State after an arbitrary number of queues (iteration ends included):
    the per-queue apply, the deg(y,C) updates and the community sums must
    leave exactly the oracle's state for the next queue."""
    el = CASES[idx]
    og = oracle_lib.OracleGraph(el.src, el.dst)
    og.set_gain_rule(RULE)
    nb = -(-og.n // q)
    points = sorted({1, 2, 3, nb - 1, nb, nb + 1, 2 * nb + 5} - {0})
    with lf.Graph(el.src, el.dst, gain_rule=RULE) as g:
        for b in points:
            og.run(q, -math.inf, 3, max_batches=b)
            g.run(q, -math.inf, 3, max_batches=b)
            compare_state(g, og)


@pytest.mark.parametrize("shape", [dict(warps_per_node=1), dict(warps_per_node=2), dict(warps_per_node=4),
                                   dict(warps_per_node=8), dict(exhaustive_fp64=True),
                                   dict(member_slots=2), dict(use_graphs=False), dict(debug_checks=True)],
                         ids=["team1", "team2", "team4", "team8", "exact_all", "row_growth", "direct_launches",
                              "bounds_checked"])
def test_literal_launch_shapes(lf, oracle_lib, shape):
    """Every team size, the bracket switched off (every candidate's gain
    summed exactly), membership rows grown from capacity 2, launches without
    graph capture, and the bounds-checked mode (no check fires) give the
    oracle's run."""
    el = W.dblp_like(seed=3, scale=0.03)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    check_run(lf, og, el, 64, -math.inf, 4, **shape)


@pytest.mark.parametrize("scale,q", [(0.05, 64), (0.05, 1024), (0.1, 1024)])
def test_literal_power_law_scaled(lf, oracle_lib, scale, q):
    """The 335k-node power-law workload at 5% and 10% of its size, at the
    queue sizes of its configuration."""
    el = W.dblp_like(scale=scale)
    check_run(lf, oracle_lib.OracleGraph(el.src, el.dst), el, q)


@pytest.mark.parametrize("make", [lambda: W.wide_fan(spokes=2100, leaves=8000, leaf_degree=60, chords=5000, seed=4),
                                  lambda: W.hub_of_triangles(12000, extra=2, seed=3)],
                         ids=["wide_fan", "hub_of_12000_triangles"])
def test_literal_hubs(lf, oracle_lib, make):
    """Nodes whose neighbours bring thousands of candidate communities take
    the block-wide, multi-part evaluation."""
    el = make()
    check_run(lf, oracle_lib.OracleGraph(el.src, el.dst), el, 256, -math.inf, 2)


def test_literal_batch(lf, oracle_lib):
    """Every graph of a batch equals the oracle run on that graph alone."""
    graphs = [W.planted_er(n=200 + 50 * i, num_comms=6, seed=i) for i in range(6)]
    graphs += [W.from_pairs(W.path(6)), W.from_pairs([(0, 1)]), W.random_graph(n=2000, m=6000, seed=9, hubs=1,
                                                                                  hub_degree=900)]
    graphs += W.batched_planted(4, seed=5, n_hi=3000)
    q = 64
    with lf.Batch(graphs, gain_rule=RULE) as b:
        b.run(q, 0.01, 50)
        info = b.info()
        comms = b.graph_communities()
    for i, el in enumerate(graphs):
        og = oracle_lib.OracleGraph(el.src, el.dst)
        ref = og.run(q, 0.01, 50, rule=RULE)
        assert info["iterations"][i] == ref["iterations"], i
        assert info["wcc_initial"][i] == ref["T0"], i
        if ref["iterations"]:
            assert info["wcc_final"][i] == ref["T"][-1], i
        assert [c.tolist() for c in comms[i]] == [c.tolist() for c in og.communities()], i


def test_literal_inserted_division(lf, oracle_lib):
    """From an inserted overlapping division (the deg(x,C) of its memberships
    are counted from scratch on the GPU)."""
    el = W.planted_er(n=400, num_comms=12, seed=8)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    _, _, labels = og.csr()
    rng = np.random.default_rng(3)
    cover = [np.sort(rng.choice(labels, size=int(rng.integers(2, 60)), replace=False)).astype(np.int32)
             for _ in range(40)]
    og.set_partition(cover)
    ref = og.run(16, 0.01, 20, rule=RULE)
    with lf.Graph(el.src, el.dst, gain_rule=RULE) as g:
        g.set_partition(cover)
        st = g.run(16, 0.01, 20)
        compare_run(st, ref)
        compare_state(g, og)


def test_literal_full_power_law_workload(lf, oracle_lib):
    """The whole 335k-node power-law workload at queue size 1024 (the oracle
    takes about half a minute)."""
    el = W.dblp_like()
    check_run(lf, oracle_lib.OracleGraph(el.src, el.dst), el, 1024)


def test_literal_is_the_default_rule(lf, oracle_lib):
    """Without a gain_rule option the library decides with the paper's gain,
    as the oracle does by default."""
    el = W.dblp_like(seed=3, scale=0.03)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    assert og.gain_rule == "literal"
    ref = og.run(64, 0.01, 50)
    with lf.Graph(el.src, el.dst) as g:
        compare_run(g.run(64, 0.01, 50), ref)
        compare_state(g, og)


def test_literal_full_power_law_workload_q64(lf, oracle_lib):
    """The whole 335k-node power-law workload at queue size 64."""
    el = W.dblp_like()
    check_run(lf, oracle_lib.OracleGraph(el.src, el.dst), el, 64)


def test_literal_edge_cases(lf, oracle_lib):
    """Empty input, self-loops and repeated pairs only, ids near the int32
    limit, max_iters = 0, and invalid arguments, with the default rule."""
    with lf.Graph(np.zeros(0, np.int32), np.zeros(0, np.int32)) as g:
        assert (g.n, g.m) == (0, 0)
        st = g.run(4, 0.01, 5)
        assert st.iterations == 1 and st.wcc_initial == 0.0
        off, mem = g.communities()
        assert off.tolist() == [0] and mem.shape[0] == 0
    big = 2**31 - 1
    src = np.array([5, 5, big, big - 7, big], np.int32)
    dst = np.array([5, 5, big - 7, big, big - 7], np.int32)
    og = oracle_lib.OracleGraph(src, dst)
    with lf.Graph(src, dst) as g:
        assert (g.n, g.m) == (2, 1)
        compare_run(g.run(1, 0.01, 10), og.run(1, 0.01, 10))
    el = W.from_pairs(W.clique(4) + [(0, 4)])
    og = oracle_lib.OracleGraph(el.src, el.dst)
    ref = og.run(1, 0.01, 0)
    with lf.Graph(el.src, el.dst) as g:
        st = g.run(1, 0.01, 0)
        assert st.iterations == 0 and st.wcc_initial == ref["T0"]
        assert [c.tolist() for c in g.community_list()] == [[0, 1, 2, 3], [4]]
    with pytest.raises(ValueError):
        lf.Graph(el.src, el.dst, gain_rule="bogus")
    with lf.Graph(el.src, el.dst) as g:
        with pytest.raises(lf.LazyFoxError):
            g.run(0, 0.01, 5)
        with pytest.raises(lf.LazyFoxError):
            g.communities()


def test_literal_bounds_checked_runs_with_hubs_and_batches(lf, oracle_lib):
    """The bounds-checked mode on the hub kernels and on a batch: no check
    fires, and the results are the oracle's."""
    el = W.hub_of_triangles(12000, extra=2, seed=3)
    check_run(lf, oracle_lib.OracleGraph(el.src, el.dst), el, 256, -math.inf, 2, debug_checks=True)
    graphs = W.batched_planted(4, seed=5, n_hi=3000)
    with lf.Batch(graphs, gain_rule=RULE, debug_checks=True) as b:
        b.run(64, 0.01, 50)
        comms = b.graph_communities()
    for i, g in enumerate(graphs):
        og = oracle_lib.OracleGraph(g.src, g.dst)
        og.run(64, 0.01, 50, rule=RULE)
        assert [c.tolist() for c in comms[i]] == [c.tolist() for c in og.communities()], i


def ring_lattice(n, k):
    """Every node joined to its k nearest neighbours on each side: all nodes
    have the same degree and the same clustering coefficient."""
    return [(i, (i + j) % n) for i in range(n) for j in range(1, k + 1)]


@pytest.mark.parametrize("q", [1, 7, 64, 1 << 30])
def test_literal_ties_everywhere(lf, oracle_lib, q):
    """Adversarial ties: a ring lattice (one CC and one degree for every node,
    so the order falls back to ids and many gains tie exactly), a complete
    bipartite graph (no triangle: cc = 0, every estimator term and total 0)
    and disjoint copies of the same clique (equal gains in every copy)."""
    graphs = [W.from_pairs(ring_lattice(60, 3), "ring_lattice_60_3"),
              W.from_pairs([(a, 10 + b) for a in range(6) for b in range(7)], "k_6_7"),
              W.from_pairs(W.clique(5) + W.clique(5, 10) + W.clique(5, 20) + [(4, 10), (14, 20)], "three_k5")]
    for el in graphs:
        og = oracle_lib.OracleGraph(el.src, el.dst)
        check_run(lf, og, el, q)


def test_literal_runs_are_deterministic(lf):
    """The FP32 corrections are summed with atomics in any order, so a
    bracket may differ in its last bits between runs; the decisions may not.
    Two runs of a power-law graph with hubs give the same totals (bit for
    bit) and the same memberships, and so does a third run with the
    bounds-checked mode on."""
    el = W.dblp_like(seed=5, scale=0.05)
    outs = []
    for kw in [{}, {}, dict(debug_checks=True)]:
        with lf.Graph(el.src, el.dst, **kw) as g:
            st = g.run(1024, -math.inf, 6)
            s = g.state()
            outs.append(([float(v).hex() for v in st.wcc_history], st.joins.tolist(), st.leaves.tolist(),
                         s["mem_off"].tolist(), s["mem_ids"].tolist()))
    assert outs[0] == outs[1] == outs[2]
