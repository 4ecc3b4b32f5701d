"""Pins of the oracle's graph preprocessing, triangle counts, node order, cc and
initial clustering against brute force, closed forms and hand-derived cases.

Paper passages: Methods > Preprocessing (Remove Multi-Edges, Dense Node
Labels, Node Order, Initial Clustering); WCC paragraph (t(x,V), vt(x,V));
Heuristic Counting of Triangles (global cc = mean of local CCs).
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2210_03211_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_simple_graph(src, dst):
    edges = set()
    for a, b in zip(src.tolist(), dst.tolist()):
        if a != b:
            edges.add((min(a, b), max(a, b)))
    ids = sorted({v for e in edges for v in e})
    return ids, edges


def brute_adj(n, edges_dense):
    nb = [set() for _ in range(n)]
    for a, b in edges_dense:
        nb[a].add(b)
        nb[b].add(a)
    return nb


def brute_triangles(nb):
    n = len(nb)
    t = [0] * n
    vt = [0] * n
    for x in range(n):
        t[x] = sum(1 for y, z in itertools.combinations(sorted(nb[x]), 2) if z in nb[y])
        vt[x] = sum(1 for y in nb[x] if nb[x] & nb[y])
    return t, vt


def small_random_cases():
    cases = []
    for seed in range(8):
        el = W.random_graph(n=30 + 3 * seed, m=90 + 10 * seed, seed=seed, self_loops=3, duplicates=10)
        cases.append(el)
    cases.append(W.random_graph(n=25, m=60, seed=99, hubs=2, hub_degree=20))
    return cases


@pytest.mark.parametrize("el", small_random_cases(), ids=lambda e: e.name)
def test_preprocess_matches_brute_force(oracle_lib, el):
    g = oracle_lib.OracleGraph(el.src, el.dst, prepare=False)
    ids, edges = brute_simple_graph(el.src, el.dst)
    off, adj, labels = g.csr()
    assert labels.tolist() == ids
    assert g.m == len(edges)
    pos = {v: i for i, v in enumerate(ids)}
    nb = brute_adj(len(ids), [(pos[a], pos[b]) for a, b in edges])
    for x in range(len(ids)):
        row = adj[off[x]:off[x + 1]].tolist()
        assert row == sorted(nb[x])


@pytest.mark.parametrize("el", small_random_cases(), ids=lambda e: e.name)
def test_triangles_match_brute_force(oracle_lib, el):
    g = oracle_lib.OracleGraph(el.src, el.dst)
    off, adj, _ = g.csr()
    nb = [set(adj[off[x]:off[x + 1]].tolist()) for x in range(g.n)]
    t_ref, vt_ref = brute_triangles(nb)
    t, vt, _ = g.node_stats()
    assert t.tolist() == t_ref
    assert vt.tolist() == vt_ref
    ntri = sum(1 for a, b, c in itertools.combinations(range(g.n), 3)
               if b in nb[a] and c in nb[a] and c in nb[b])
    assert int(t.sum()) == 3 * ntri
    assert np.all(vt <= off[1:] - off[:-1])
    for x in range(g.n):
        assert g.node_triangles(x) == (t_ref[x], vt_ref[x])


@pytest.mark.parametrize("k", [3, 4, 5, 9])
def test_closed_forms_clique(oracle_lib, k):
    el = W.from_pairs(W.clique(k))
    g = oracle_lib.OracleGraph(el.src, el.dst)
    t, vt, cc = g.node_stats()
    assert t.tolist() == [math.comb(k - 1, 2)] * k
    assert vt.tolist() == [k - 1] * k
    assert cc == 1.0


def test_closed_forms_star_cycle_wheel(oracle_lib):
    g = oracle_lib.OracleGraph(*(lambda e: (e.src, e.dst))(W.from_pairs(W.star(7))))
    t, vt, cc = g.node_stats()
    assert t.sum() == 0 and vt.sum() == 0 and cc == 0.0
    for k in (4, 5, 11):
        e = W.from_pairs(W.cycle(k))
        g = oracle_lib.OracleGraph(e.src, e.dst)
        t, vt, cc = g.node_stats()
        assert t.sum() == 0 and vt.sum() == 0
    e = W.from_pairs(W.cycle(3))
    g = oracle_lib.OracleGraph(e.src, e.dst)
    assert g.node_stats()[0].tolist() == [1, 1, 1]
    # wheel: hub 0 joined to a rim cycle 1..k; hub in k triangles, rim nodes in 2
    k = 8
    rim = [(1 + i, 1 + (i + 1) % k) for i in range(k)]
    e = W.from_pairs(rim + [(0, 1 + i) for i in range(k)])
    g = oracle_lib.OracleGraph(e.src, e.dst)
    t, vt, cc = g.node_stats()
    assert t.tolist() == [k] + [2] * k
    assert vt.tolist() == [k] + [3] * k
    # CC: hub k / C(k,2), rim 2 / C(3,2); cc is their exact mean, rounded
    exact = (Fraction(k, math.comb(k, 2)) + k * Fraction(2, 3)) / (k + 1)
    assert abs(cc - float(exact)) <= 2 * math.ulp(float(exact))


@pytest.mark.parametrize("el", small_random_cases()[:5] + [W.eu_core_like()], ids=lambda e: e.name)
def test_order_and_cc_match_fractions(oracle_lib, el):
    g = oracle_lib.OracleGraph(el.src, el.dst)
    off, _, _ = g.csr()
    d = (off[1:] - off[:-1]).tolist()
    t, _, cc = g.node_stats()
    t = t.tolist()

    def ccf(x):
        return Fraction(t[x], d[x] * (d[x] - 1) // 2) if d[x] > 1 else Fraction(0)

    ref = sorted(range(g.n), key=lambda x: (-ccf(x), -d[x], x))
    assert g.order().tolist() == ref
    # cc = RN( RN(sum of rounded local CCs) / n ); Python's float(Fraction) rounds correctly
    rounded = [t[x] / (d[x] * (d[x] - 1) // 2) if d[x] > 1 else 0.0 for x in range(g.n)]
    s = float(sum(Fraction(v) for v in rounded))
    assert cc == s / g.n
    assert 0.0 <= cc <= 1.0


def lexfirst_mis_ok(order, nb, seeds):
    pos = {x: i for i, x in enumerate(order)}
    for x in order:
        earlier_seed = any(pos[y] < pos[x] and y in seeds for y in nb[x])
        if (x in seeds) == earlier_seed:
            return False
    return True


@pytest.mark.parametrize("el", small_random_cases() + [W.eu_core_like()], ids=lambda e: e.name)
def test_initial_clustering_is_greedy_in_order(oracle_lib, el):
    """Initial Clustering: the openers form the lexicographically-first maximal
    independent set in the node order (a node opens a community iff no earlier
    neighbour opened one), ids follow opening order, and every other node sits
    in the community of its earliest opening neighbour."""
    g = oracle_lib.OracleGraph(el.src, el.dst)
    g.init_clustering()
    off, adj, _ = g.csr()
    nb = [set(adj[off[x]:off[x + 1]].tolist()) for x in range(g.n)]
    order = g.order().tolist()
    pos = {x: i for i, x in enumerate(order)}
    s = g.state()
    comm = [s["mem_ids"][s["mem_off"][x]:s["mem_off"][x + 1]].tolist() for x in range(g.n)]
    assert all(len(c) == 1 for c in comm)
    comm = [c[0] for c in comm]
    k = len(s["n"])
    # the opener of community c is its member with the earliest position
    opener = {}
    for x in order:
        opener.setdefault(comm[x], x)
    seeds = set(opener.values())
    assert lexfirst_mis_ok(order, nb, seeds)
    assert sorted(opener.keys(), key=lambda c: pos[opener[c]]) == list(range(k))
    for x in range(g.n):
        if x in seeds:
            continue
        first = min((y for y in nb[x] if y in seeds), key=lambda y: pos[y])
        assert comm[x] == comm[first]
    # aggregates equal recounts
    for c in range(k):
        members = [x for x in range(g.n) if comm[x] == c]
        assert s["n"][c] == len(members)
        assert s["vol"][c] == sum(len(nb[x]) for x in members)
        ms = set(members)
        assert s["m"][c] == sum(1 for x in members for y in nb[x] if y in ms and y > x)


def test_disjoint_cliques_initial_clustering(oracle_lib):
    pairs = W.clique(5, 0) + W.clique(4, 10) + W.clique(7, 20)
    el = W.from_pairs(pairs)
    g = oracle_lib.OracleGraph(el.src, el.dst)
    g.init_clustering()
    _, _, labels = g.csr()
    s = g.state()
    groups = {}
    for x in range(g.n):
        for c in s["mem_ids"][s["mem_off"][x]:s["mem_off"][x + 1]]:
            groups.setdefault(int(c), []).append(int(labels[x]))
    got = sorted(sorted(v) for v in groups.values())
    assert got == sorted([list(range(0, 5)), list(range(10, 14)), list(range(20, 27))])


@pytest.mark.parametrize("name", ["bowtie", "k4_pendant", "path5", "triangle_tail"])
def test_golden_preprocessing(oracle_lib, name):
    fx = json.load(open(os.path.join(GOLDEN, name + ".json")))
    el = W.from_pairs(fx["edges"])
    g = oracle_lib.OracleGraph(el.src, el.dst)
    t, vt, cc = g.node_stats()
    assert t.tolist() == fx["t"]
    assert vt.tolist() == fx["vt"]
    assert abs(cc - float(Fraction(fx["cc"]))) <= math.ulp(1.0)
    assert g.order().tolist() == fx["order"]
    g.init_clustering()
    s = g.state()
    groups = {}
    for x in range(g.n):
        for c in s["mem_ids"][s["mem_off"][x]:s["mem_off"][x + 1]]:
            groups.setdefault(int(c), []).append(x)
    assert [groups[c] for c in sorted(groups)] == fx["init_communities"]
    assert s["n"].tolist() == fx["init_n"]
    assert s["m"].tolist() == fx["init_m"]
    assert s["vol"].tolist() == fx["init_vol"]


def test_rejects_negative_ids(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.OracleGraph(np.array([0, -1], np.int32), np.array([1, 2], np.int32))


def test_empty_and_self_loops_only(oracle_lib):
    g = oracle_lib.OracleGraph(np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert (g.n, g.m) == (0, 0)
    g = oracle_lib.OracleGraph(np.array([3, 3, 5], np.int32), np.array([3, 3, 5], np.int32))
    assert (g.n, g.m) == (0, 0)
    r = g.run(4, 0.01, 5)
    assert r["iterations"] == 1 and r["T0"] == 0.0
