"""Pins of the oracle's inserted division (Methods, Initial Clustering: an
existing division may replace the initial clustering) and of resuming from
the communities saved after an iteration (the per-iteration results the paper
writes to disk on Friendster)."""
import math

import numpy as np
import pytest

from paper_2210_03211_gb300 import workloads as W


def _recount(og, comms):
    """n_C, internal edges m_C and vol_C of a cover, by brute force."""
    off, adj, labels = og.csr()
    deg = np.diff(off)
    pos = {int(l): i for i, l in enumerate(labels)}
    out = []
    for c in comms:
        xs = sorted(pos[int(v)] for v in c)
        S = set(xs)
        m = sum(1 for x in xs for y in adj[off[x]:off[x + 1]] if y > x and int(y) in S)
        out.append((len(xs), m, int(sum(deg[x] for x in xs))))
    return out


def test_inserted_initial_clustering_reproduces_the_run(oracle_lib):
    """The initial clustering, taken out and inserted again, gives the same run
    bit for bit (so the inserted state is exactly the one the clustering
    builds: same ids, same aggregates)."""
    el = W.eu_core_like()
    g = oracle_lib.OracleGraph(el.src, el.dst)
    g.run(16, 0.01, 0)
    init = g.communities()
    ref = g.run(16, 0.01, 50)
    ref_state = g.state()
    g2 = oracle_lib.OracleGraph(el.src, el.dst)
    g2.set_partition(init)
    out = g2.run(16, 0.01, 50)
    assert out["T0"] == ref["T0"] and out["iterations"] == ref["iterations"]
    assert np.array_equal(out["T"], ref["T"])
    assert np.array_equal(out["joins"], ref["joins"]) and np.array_equal(out["leaves"], ref["leaves"])
    s = g2.state()
    for key in ("mem_off", "mem_ids", "n", "m", "vol"):
        assert np.array_equal(s[key], ref_state[key]), key


@pytest.mark.parametrize("q,a,b", [(1, 2, 3), (64, 1, 4), (1 << 20, 3, 2)])
def test_resume_from_saved_communities_equals_one_run(oracle_lib, q, a, b):
    """Run a iterations, save the communities, insert them and run b more: the
    same totals, moves and final communities as a + b iterations in one run."""
    el = W.random_graph(n=300, m=1800, seed=7, hubs=2, hub_degree=60)
    full = oracle_lib.OracleGraph(el.src, el.dst)
    ref = full.run(q, -math.inf, a + b)
    g = oracle_lib.OracleGraph(el.src, el.dst)
    first = g.run(q, -math.inf, a)
    saved = g.communities()
    g.set_partition(saved)
    second = g.run(q, -math.inf, b)
    assert second["T0"] == first["T"][-1] == ref["T"][a - 1]
    assert np.array_equal(np.concatenate([first["T"], second["T"]]), ref["T"])
    assert np.array_equal(np.concatenate([first["joins"], second["joins"]]), ref["joins"])
    assert np.array_equal(np.concatenate([first["leaves"], second["leaves"]]), ref["leaves"])
    assert [c.tolist() for c in g.communities()] == [c.tolist() for c in full.communities()]


def test_inserted_cover_aggregates_equal_brute_force(oracle_lib):
    """An overlapping cover (the planted one, plus a community spanning
    several of them): n_C, m_C, vol_C equal a brute-force recount, and every
    node's row lists its communities in ascending id."""
    el = W.eu_core_like()
    comms = [np.asarray(c, dtype=np.int32) for c in el.planted]
    comms.append(np.unique(np.concatenate([comms[0][:5], comms[1][:5], comms[2][:5]])))
    g = oracle_lib.OracleGraph(el.src, el.dst)
    _, _, labels = g.csr()
    comms = [c[np.isin(c, labels)] for c in comms]
    g.set_partition(comms)
    g.run(1, 0.01, 0)
    s = g.state()
    want = _recount(g, comms)
    assert [(int(s["n"][c]), int(s["m"][c]), int(s["vol"][c])) for c in range(len(comms))] == want
    for x in range(g.n):
        row = s["mem_ids"][s["mem_off"][x]:s["mem_off"][x + 1]]
        assert np.all(np.diff(row) > 0)
    g.set_check_invariants(True)
    g.run(1, 0.01, 3)
    assert g.invariant_failures() == 0


def test_invalid_divisions_are_rejected(oracle_lib):
    el = W.from_pairs(W.clique(4) + [(3, 10)], "k4_tail")
    g = oracle_lib.OracleGraph(el.src, el.dst)
    with pytest.raises(ValueError):
        g.set_partition([np.array([0, 1, 99], dtype=np.int32)])   # 99 is not a node
    with pytest.raises(ValueError):
        g.set_partition([np.array([0, 1, 1], dtype=np.int32)])    # 1 twice in one community
    g.set_partition([np.array([0, 1], dtype=np.int32), np.array([1, 2, 3, 10], dtype=np.int32)])
    g.set_partition(None)   # back to the initial clustering
    a = g.run(1, 0.01, 5)
    b = oracle_lib.OracleGraph(el.src, el.dst).run(1, 0.01, 5)
    assert np.array_equal(a["T"], b["T"])


@pytest.mark.parametrize("rule", ["literal", "meanfield"])
def test_golden_leave_from_an_inserted_division(oracle_lib, rule):
    """A hand-derived run with a leave (tests/golden/pendant_leave.json): the
    pendant node of an inserted division leaves it, and the mean-field and
    literal gains of the start's moves have the hand values; the run is the
    same under both rules."""
    import json
    import os
    from fractions import Fraction
    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pendant_leave.json")))
    assert rule in fx["gain_rules"]
    el = W.from_pairs(fx["edges"])
    g = oracle_lib.OracleGraph(el.src, el.dst)
    assert g.cc == pytest.approx(float(Fraction(fx["cc"])), rel=2 ** -52)
    g.set_partition([np.array(c, np.int32) for c in fx["partition"]])
    g.run(fx["queue_size"], fx["threshold"], 0, rule="meanfield")
    eps = 2.0 ** -52
    ev = g.evaluate(3)
    assert ev["leave"] == 0 and ev["join"] == -1 and ev["kleave"] == 1
    assert abs(ev["gleave"] - float(Fraction(fx["leave_gain_node3"]))) <= 8 * eps * 64 / 21
    assert abs(g.literal_gain(3, 0) - float(Fraction(fx["literal_leave_gain_node3"]))) <= 8 * eps * 4
    for x, c, want in fx["literal_gains_at_start"]:
        assert abs(g.literal_gain(x, c) - float(Fraction(want))) <= 16 * eps * 4, (x, c)
    r = g.run(fx["queue_size"], fx["threshold"], fx["max_iters"], rule=rule)
    assert r["T0"] == pytest.approx(float(Fraction(fx["T0"])), rel=1e-14)
    assert r["iterations"] == fx["iterations"] and r["converged"]
    for got, want in zip(r["T"], fx["T"]):
        assert got == pytest.approx(float(Fraction(want)), rel=1e-14)
    assert r["joins"].tolist() == fx["joins"] and r["leaves"].tolist() == fx["leaves"]
    assert [c.tolist() for c in g.communities()] == fx["final_communities"]
