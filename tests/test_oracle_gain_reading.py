"""Pins of the paper's gain and of the diagnostic that compares the two gain
rules.  The literal gain -- the change of the paper's \\wcchat(P), the sum of
the per-node estimator over all memberships (Joining / Leaving a Community)
-- decides runs by default; the mean-field departure scores a community from
its aggregates alone.  The diagnostic takes every decision with both rules on
the same snapshot and counts how often they agree.  The literal gain is
pinned here to differences of the oracle's own totals on inserted covers
(Methods, Initial Clustering: inserted divisions), to a hand derivation on
the bowtie, and to a brute-force choice."""
import math

import numpy as np
import pytest

from paper_2210_03211_gb300 import workloads as W

EPS = 2.0 ** -52


def _cover(og):
    """Live communities as {community id: sorted dense ids}."""
    s = og.state()
    out = {int(c): [] for c in np.flatnonzero(s["n"] > 0)}
    for x in range(og.n):
        for c in s["mem_ids"][s["mem_off"][x]:s["mem_off"][x + 1]]:
            out[int(c)].append(x)
    return out


def _total_of(oracle_lib, el, labels, cover):
    """\\wcchat(P) of a cover (dense ids), through a fresh graph with the cover inserted."""
    g = oracle_lib.OracleGraph(el.src, el.dst)
    g.set_partition([labels[np.asarray(v, dtype=np.int64)] for v in cover.values() if len(v)])
    return g.run(1, 0.01, 0)["T0"]


def _moved(cover, x, c):
    out = {k: list(v) for k, v in cover.items()}
    if x in out[c]:
        out[c].remove(x)
    else:
        out[c] = sorted(out[c] + [x])
    return out


def _candidates(og, cover, x):
    off, adj, _ = og.csr()
    own = {c for c, v in cover.items() if x in v}
    met = {c for c, v in cover.items() for y in adj[off[x]:off[x + 1]] if int(y) in v}
    return sorted(met - own), sorted(own)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_literal_gain_equals_the_change_of_the_total(oracle_lib, seed):
    el = W.planted_er(n=60, num_comms=5, size_lo=8, size_hi=20, p_in=0.35, seed=seed)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    og.run(1, -math.inf, 2)
    _, _, labels = og.csr()
    cover = _cover(og)
    base = _total_of(oracle_lib, el, labels, cover)
    checked = 0
    for x in range(0, og.n, 3):
        joins, leaves = _candidates(og, cover, x)
        for c in joins[:2] + leaves[:2]:
            lit = og.literal_gain(x, c)
            after = _total_of(oracle_lib, el, labels, _moved(cover, x, c))
            assert abs(lit - (after - base)) <= 8 * EPS * max(abs(base), abs(after), 1.0), (x, c)
            checked += 1
    assert checked > 20


def test_literal_gain_on_the_bowtie_by_hand(oracle_lib):
    """Bowtie (two triangles sharing node 2), initial clustering {0,1,2}, {3,4};
    cc = 13/15.  Node 2 joining {3,4}: the members' terms rise from 0 (one
    neighbour inside, C(1,2) = 0) to (15/13)(2/2) each, and node 2 adds
    (1/(6*13/15))(4/4) = 5/26: gain 65/26 -- the whole change of the total in
    the first iteration, where it is the only move.  Node 2 leaving {0,1,2}:
    the three terms 15/13, 15/13, 5/26 drop to 0 (a pair keeps C(1,2) = 0):
    gain -65/26."""
    og = oracle_lib.OracleGraph(np.array([0, 0, 1, 2, 2, 3], np.int32), np.array([1, 2, 2, 3, 4, 4], np.int32))
    og.run(1, 0.01, 0)
    assert abs(og.cc - 13 / 15) <= EPS
    assert abs(og.literal_gain(2, 1) - 65 / 26) <= 4 * EPS * 3
    assert abs(og.literal_gain(2, 0) + 65 / 26) <= 4 * EPS * 3
    d = og.evaluate_literal(2)
    assert d["join"] == 1 and d["leave"] == -1
    assert abs(d["gjoin"] - 65 / 26) <= 4 * EPS * 3


def test_literal_decision_by_brute_force(oracle_lib):
    """Every node's literal decision equals the best strictly positive change
    of the total over its candidates (ties to the lowest id), with each change
    taken from the totals of inserted covers; gains within rounding distance
    of each other or of 0 are not decided here."""
    el = W.planted_er(n=40, num_comms=4, size_lo=6, size_hi=14, p_in=0.4, seed=7)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    og.run(1, -math.inf, 1)
    _, _, labels = og.csr()
    cover = _cover(og)
    base = _total_of(oracle_lib, el, labels, cover)
    tol = 16 * EPS * max(abs(base), 1.0)
    decided = 0
    for x in range(og.n):
        joins, leaves = _candidates(og, cover, x)
        d = og.evaluate_literal(x)
        for kind, cands in (("join", joins), ("leave", leaves)):
            gains = [(_total_of(oracle_lib, el, labels, _moved(cover, x, c)) - base, c) for c in cands]
            pos = [(g, c) for g, c in gains if g > tol]
            if any(abs(g) <= tol for g, _ in gains):
                continue
            if not pos:
                assert d[kind] == -1, (x, kind, gains)
            else:
                best = max(g for g, _ in pos)
                if sum(1 for g, _ in pos if best - g <= tol) > 1:
                    continue
                assert d[kind] == next(c for g, c in pos if g == best), (x, kind, gains)
            decided += 1
    assert decided > og.n


def test_diagnostic_sees_the_run_decisions(oracle_lib):
    el = W.planted_er(n=120, num_comms=6, size_lo=10, size_hi=30, p_in=0.3, seed=3)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    og.set_literal_diagnostic(True)
    r = og.run(4, 0.01, 50, rule="meanfield")
    d = og.literal_diagnostic()
    assert d["evaluations"] == og.n * r["iterations"]
    assert d["joins_meanfield"] == int(r["joins"].sum())
    assert d["leaves_meanfield"] == int(r["leaves"].sum())
    assert d["same_both"] <= min(d["same_join"], d["same_leave"]) <= d["evaluations"]
    # the diagnostic changes nothing in the run
    og.set_literal_diagnostic(False)
    r2 = og.run(4, 0.01, 50, rule="meanfield")
    assert r2["iterations"] == r["iterations"] and np.array_equal(r2["T"], r["T"])
    assert og.literal_diagnostic()["evaluations"] == 0


def test_disjoint_cliques_agree_completely(oracle_lib):
    """Isolated cliques: no join candidate outside a node's own clique and
    leaving lowers both scores, so neither reading moves a node."""
    src, dst = [], []
    for base, k in ((0, 4), (10, 5), (20, 6)):
        for i in range(k):
            for j in range(i + 1, k):
                src.append(base + i)
                dst.append(base + j)
    og = oracle_lib.OracleGraph(np.array(src, np.int32), np.array(dst, np.int32))
    og.set_literal_diagnostic(True)
    og.run(1, 0.01, 5)
    d = og.literal_diagnostic()
    assert d["evaluations"] == og.n and d["same_both"] == og.n
    assert d["joins_literal"] == d["leaves_literal"] == 0


def test_meanfield_history_is_the_sum_of_community_scores(oracle_lib):
    """The diagnostic history beside the literal totals: after every
    iteration, the correctly rounded sum of S(n_C, m_C, vol_C) over the live
    communities -- checked on the last iteration against the scores of the
    final aggregates, and on isolated cliques against the closed form
    S = n / cc (every member's estimator is 1/cc there)."""
    el = W.planted_er(n=120, num_comms=6, size_lo=10, size_hi=30, p_in=0.3, seed=3)
    og = oracle_lib.OracleGraph(el.src, el.dst)
    r = og.run(4, 0.01, 50)
    assert r["S"].shape == r["T"].shape
    st = og.state()
    terms = [oracle_lib.community_score(int(n), int(m), int(v), og.cc)
             for n, m, v in zip(st["n"], st["m"], st["vol"]) if n > 0]
    assert r["S"][-1] == oracle_lib.fsum(terms)
    src, dst = [], []
    for base, k in ((0, 4), (10, 5), (20, 6)):
        for i in range(k):
            for j in range(i + 1, k):
                src.append(base + i)
                dst.append(base + j)
    og = oracle_lib.OracleGraph(np.array(src, np.int32), np.array(dst, np.int32))
    r = og.run(1, 0.01, 5)
    assert og.cc == 1.0 and abs(r["S"][-1] - 15.0) <= 8 * EPS * 15 and abs(r["T"][-1] - 15.0) <= 8 * EPS * 15
