"""Serving with continuous batching (lf_server_*): jobs submitted while others
run are admitted as slots and the memory budget allow, run side by side, and
each job's result is the one the same graph gives alone."""
import math

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


def jobs():
    gs = W.batched_planted(10, seed=13, n_lo=500, n_hi=20000)
    gs.append(W.random_graph(n=3000, m=9000, seed=12, hubs=2, hub_degree=2600))
    gs.append(W.dblp_like(seed=3, scale=0.03))
    return gs


def alone(lf, el, q, thr, it):
    with lf.Graph(el.src, el.dst) as g:
        g.run(q, thr, it)
        return [c.tolist() for c in g.community_list()]


@pytest.mark.parametrize("q", [64, 256])
def test_results_in_the_mix_equal_alone(lf, q):
    graphs = jobs()
    with lf.Server(hbm_budget_bytes=8 << 30, max_active=4) as srv:
        ids = [srv.submit(el.src, el.dst, q, 0.01, 50) for el in graphs]
        res = [srv.wait(j) for j in ids]
        comms = [[c.tolist() for c in srv.community_list(j)] for j in ids]
    for el, r, c in zip(graphs, res, comms):
        assert r["status"] == lf.LF_OK
        assert c == alone(lf, el, q, 0.01, 50)
    # jobs overlapped on the device: some job was admitted before another finished
    spans = sorted((r["t_admit_ms"], r["t_done_ms"]) for r in res)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    assert all(r["t_submit_ms"] <= r["t_admit_ms"] <= r["t_done_ms"] for r in res)


def test_budget_admits_one_job_at_a_time(lf):
    graphs = jobs()[:5]
    with lf.Server(hbm_budget_bytes=1, max_active=4) as srv:
        ids = [srv.submit(el.src, el.dst, 256, 0.01, 50) for el in graphs]
        res = [srv.wait(j) for j in ids]
    spans = sorted((r["t_admit_ms"], r["t_done_ms"]) for r in res)
    assert all(spans[i + 1][0] >= spans[i][1] for i in range(len(spans) - 1))


def test_oracle_parity_through_the_server(lf, oracle_lib):
    graphs = jobs()[:3]
    with lf.Server(max_active=3) as srv:
        ids = [srv.submit(el.src, el.dst, 16, -math.inf, 4) for el in graphs]
        for el, j in zip(graphs, ids):
            r = srv.wait(j)
            og = oracle_lib.OracleGraph(el.src, el.dst)
            ref = og.run(16, -math.inf, 4)
            assert r["iterations"] == ref["iterations"]
            assert r["wcc_final"] == ref["T"][-1]
            assert [c.tolist() for c in srv.community_list(j)] == [c.tolist() for c in og.communities()]


def test_a_failing_job_does_not_stop_the_server(lf):
    good = jobs()[0]
    with lf.Server(max_active=2) as srv:
        bad = srv.submit(np.array([0, 1], np.int32), np.array([1, -5], np.int32), 16, 0.01, 5)
        ok = srv.submit(good.src, good.dst, 16, 0.01, 5)
        with pytest.raises(lf.LazyFoxError) as e:
            srv.wait(bad)
        assert e.value.status == lf.LF_ERR_INVALID
        assert srv.wait(ok)["status"] == lf.LF_OK


def test_destroy_cancels_jobs_not_yet_admitted(lf):
    import threading
    import time
    el = W.dblp_like(seed=3, scale=0.3)
    srv = lf.Server(max_active=1)
    ids = [srv.submit(el.src, el.dst, 16, -math.inf, 20) for _ in range(6)]
    out = {}

    def waiter():
        try:
            out["res"] = srv.wait(ids[-1])
        except lf.LazyFoxError as e:
            out["err"] = e

    t = threading.Thread(target=waiter)
    t.start()
    time.sleep(0.3)   # the waiter is inside lf_server_wait; the first job (20 full iterations) still runs
    srv.close()       # returns once the running job finished and the waiter left
    t.join(60)
    assert not t.is_alive()
    assert "err" in out, out
    assert out["err"].status == lf.LF_ERR_STATE and "cancelled" in str(out["err"])


def test_admission_estimate_bounds_each_jobs_device_memory(lf):
    """The memory the server reserves for a job (est_bytes, from its edge
    count) is at least the device memory the same graph's run actually
    holds at its peak (counted through the allocation callbacks); with the
    admission rule (reserved estimates within the budget) the jobs resident
    at any time therefore fit the budget.  Graphs of the serving workload's
    shape (planted, average degree 10-80), a hub graph and the power-law
    workload at 10%."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    graphs = W.serving_jobs(10, seed=7, n_hi=60000)[0]
    graphs += [W.random_graph(n=3000, m=9000, seed=12, hubs=2, hub_degree=2600), W.dblp_like(scale=0.1)]
    with lf.Server(max_active=2) as srv:
        est = [srv.wait(srv.submit(el.src, el.dst, 1024, 0.01, 50))["est_bytes"] for el in graphs]
    for el, e in zip(graphs, est):
        a = lf.CountingAllocator(dev)
        with lf.Graph(el.src, el.dst, allocator=a) as g:
            g.run(1024, 0.01, 50)
            g.communities()
        assert 0 < a.peak <= e, (len(el.src), a.peak, e)


def test_resident_estimates_stay_within_the_budget(lf):
    """Jobs overlapping in time never reserve more than the budget together
    (a job larger than the whole budget runs alone)."""
    graphs = jobs()
    budget = 3 * max(228 * len(el.src) + (64 << 20) for el in graphs) // 2
    with lf.Server(hbm_budget_bytes=budget, max_active=4) as srv:
        ids = [srv.submit(el.src, el.dst, 256, 0.01, 50) for el in graphs]
        res = [srv.wait(j) for j in ids]
    for r in res:
        others = [o for o in res if o is not r and o["t_admit_ms"] < r["t_done_ms"] and r["t_admit_ms"] < o["t_done_ms"]]
        overlapping = r["est_bytes"] + sum(o["est_bytes"] for o in others if o["t_admit_ms"] <= r["t_admit_ms"])
        assert r["est_bytes"] > budget or overlapping <= budget, (r, budget)
