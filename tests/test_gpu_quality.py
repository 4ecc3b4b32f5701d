"""F1-score of overlapping covers on the GPU (lf_cover_f1) against the
oracle, bit for bit, and the quality report (LazyFox against Fox and against
the planted cover, as in the paper's quality table)."""
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


def random_cover(rng, k, n, lo, hi):
    return [np.unique(rng.integers(0, n, rng.integers(lo, hi))).astype(np.int32) for _ in range(k)]


@pytest.mark.parametrize("seed,k,n,lo,hi", [(1, 30, 200, 2, 20), (2, 500, 5000, 5, 60), (3, 40, 3000, 200, 3000)])
def test_cover_f1_equals_oracle(lf, oracle_lib, seed, k, n, lo, hi):
    rng = np.random.default_rng(seed)
    det, ref = random_cover(rng, k, n, lo, hi), random_cover(rng, k + 7, n, lo, hi)
    f, best = lf.cover_f1(det, ref)
    of, obest = oracle_lib.cover_f1(det, ref)
    assert f == of
    assert np.array_equal(best, obest)


def test_many_candidates_need_several_passes(lf, oracle_lib):
    """One detected community over 6,000 nodes, each in its own reference
    community and in a shared one: more candidates than one table pass."""
    ref = [np.array([i], dtype=np.int32) for i in range(6000)] + [np.arange(0, 6000, 3, dtype=np.int32)]
    det = [np.arange(6000, dtype=np.int32), np.arange(10, 20, dtype=np.int32)]
    f, best = lf.cover_f1(det, ref)
    of, obest = oracle_lib.cover_f1(det, ref)
    assert f == of and np.array_equal(best, obest)


def test_detected_communities_against_planted_and_fox(lf, oracle_lib):
    el = W.eu_core_like()
    og = oracle_lib.OracleGraph(el.src, el.dst)
    og.run(1, 0.01, 50)
    fox = og.communities()
    og.run(64, 0.01, 50)
    lazy = og.communities()
    planted = [np.unique(np.asarray(c, dtype=np.int32)) for c in el.planted]
    for det, ref in ((lazy, fox), (lazy, planted), (fox, planted)):
        assert lf.cover_f1(det, ref)[0] == oracle_lib.cover_f1(det, ref)[0]
    rows = lf.quality_report(el, queue_sizes=(2, 64))
    assert rows[0]["queue_size"] == 1 and rows[0]["f1_vs_fox"] == 1.0
    assert rows[2]["f1_vs_fox"] == oracle_lib.cover_f1(lazy, fox)[0]
    assert rows[2]["f1_vs_planted"] == oracle_lib.cover_f1(lazy, planted)[0]


def test_invalid_covers(lf):
    with pytest.raises(lf.LazyFoxError):
        lf.cover_f1([np.array([], np.int32)], [np.array([1], np.int32)])   # empty community
    with pytest.raises(lf.LazyFoxError):
        lf.cover_f1([np.array([-1, 2], np.int32)], [np.array([1], np.int32)])
    assert lf.cover_f1([], [np.array([1], np.int32)])[0] == 0.0
