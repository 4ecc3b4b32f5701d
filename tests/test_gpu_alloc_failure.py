"""A device allocation that fails, at every point of graph creation and of a
run: the call reports LF_ERR_OOM, nothing stays allocated once the handle is
gone, and a run after a failed one gives the result of a clean run.  The
failure is injected on the host (the allocation callback returns NULL, as a
failing allocator would); no kernel is made to fault."""
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


CASES = [
    # planted communities, the paper's gain, per-queue launches
    (lambda: W.planted_er(n=300, num_comms=10, seed=3), 16, "literal"),
    # a graph with hubs (the hub kernels and global tables), the paper's gain
    (lambda: W.random_graph(n=3000, m=9000, seed=12, hubs=2, hub_degree=2600), 512, "literal"),
    # the mean-field rule with the persistent queue kernel
    (lambda: W.planted_er(n=300, num_comms=10, seed=3), 16, "meanfield"),
]


@pytest.mark.parametrize("make,q,rule", CASES, ids=["planted_literal", "hubs_literal", "planted_meanfield"])
def test_allocation_failure_at_every_step(lf, make, q, rule):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    el = make()
    clean = lf.CountingAllocator(dev)
    with lf.Graph(el.src, el.dst, allocator=clean, gain_rule=rule) as g:
        ref = g.run(q, 0.01, 50)
        total = clean.calls   # allocations of the creation and the run
        ref_comms = [c.tolist() for c in g.community_list()]
    assert clean.live == 0
    assert total > 10
    failed_create = failed_run = 0
    for k in range(1, total + 1):
        a = lf.CountingAllocator(dev, fail_at=k)
        try:
            g = lf.Graph(el.src, el.dst, allocator=a, gain_rule=rule)
        except lf.LazyFoxError as e:
            assert e.status == lf.LF_ERR_OOM, (k, str(e))
            assert a.live == 0, k   # the failed creation released everything
            failed_create += 1
            continue
        with g:
            try:
                st = g.run(q, 0.01, 50)
            except lf.LazyFoxError as e:
                assert e.status == lf.LF_ERR_OOM, (k, str(e))
                with pytest.raises(lf.LazyFoxError):
                    g.communities()   # no result after a failed run
                failed_run += 1
                st = g.run(q, 0.01, 50)   # the allocator no longer fails: a clean run
            assert st.iterations == ref.iterations and np.array_equal(st.wcc_history, ref.wcc_history), k
            assert [c.tolist() for c in g.community_list()] == ref_comms, k
        assert a.live == 0, k
    assert failed_create > 0 and failed_run > 0
