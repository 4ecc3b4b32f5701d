"""Pins of the seeded synthetic workloads that every parity test and every
recorded number depends on: the counter-based splitmix64 stream against its
published definition (computed here with Python integers), determinism, and
the sizes of the workloads the benchmark and the quality table are quoted on."""
import numpy as np
import pytest

from paper_2210_03211_gb300 import workloads as W

MASK = (1 << 64) - 1
GOLDEN, M1, M2 = 0x9E3779B97F4A7C15, 0xBF58476D1CE4E5B9, 0x94D049BB133111EB


def mix64(z: int) -> int:
    """splitmix64's output function (Steele, Lea and Flood 2014), Python integers."""
    z = ((z ^ (z >> 30)) * M1) & MASK
    z = ((z ^ (z >> 27)) * M2) & MASK
    return z ^ (z >> 31)


def test_stream_follows_the_splitmix64_definition():
    """Draw i of stream (seed, s) is mix64(key + (i + 1) * golden) with
    key = mix64(seed + s * golden), all modulo 2^64."""
    for seed, sid in ((0, 1), (5, 31), (123456789, 37), (2 ** 63 + 11, 2)):
        key = mix64((seed + sid * GOLDEN) & MASK)
        st = W.Stream(seed, sid)
        got = st.u64(5).tolist() + st.u64(3).tolist()   # the counter carries over between calls
        want = [mix64((key + (i + 1) * GOLDEN) & MASK) for i in range(8)]
        assert got == want
    # the textbook first output of splitmix64 seeded with 0 (state advanced by golden once)
    assert mix64(GOLDEN) == 0xE220A8397B1DCDAF


def test_stream_maps():
    st = W.Stream(9, 3)
    u = W.Stream(9, 3).u64(1000)
    x = st.integers(10, 20, 1000)
    assert np.array_equal(x, 10 + (((u >> np.uint64(32)) * np.uint64(10)) >> np.uint64(32)).astype(np.int64))
    f = W.Stream(9, 3).uniform(1000)
    assert np.all((f >= 0) & (f < 1))
    assert np.array_equal(f, (u >> np.uint64(11)).astype(np.float64) / 2.0 ** 53)
    p = W.Stream(9, 3).permutation(1000)
    assert np.array_equal(np.sort(p), np.arange(1000))


def _simple(el):
    """Nodes and undirected simple edges after dropping self-loops and repeats."""
    a = np.minimum(el.src, el.dst).astype(np.int64)
    b = np.maximum(el.src, el.dst).astype(np.int64)
    keep = a != b
    pairs = np.unique(a[keep] << 32 | b[keep])
    u, v = pairs >> 32, pairs & 0xFFFFFFFF
    nodes, inv = np.unique(np.concatenate([u, v]), return_inverse=True)
    deg = np.bincount(inv, minlength=nodes.shape[0])
    return nodes.shape[0], pairs.shape[0], int(deg.max()) if deg.size else 0


def test_same_seed_same_graph_and_seeds_differ():
    a, b, c = W.planted_er(n=300, seed=4), W.planted_er(n=300, seed=4), W.planted_er(n=300, seed=5)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)
    assert not (a.src.shape == c.src.shape and np.array_equal(a.src, c.src))


def test_eu_core_stand_in_sizes():
    el = W.eu_core_like()
    assert _simple(el)[:2] == (1000, 15801)
    assert len(el.planted) == 20


@pytest.mark.slow
def test_dblp_stand_in_sizes():
    """The benchmark's 335k-node workload: 335,000 nodes, 934,381 edges, max degree 551."""
    assert _simple(W.dblp_like()) == (335000, 934381, 551)


def test_batched_and_serving_shapes():
    gs = W.batched_planted(6, seed=5)
    for el in gs:
        n, m, _ = _simple(el)
        assert 100 <= n <= 20000 and m > 0
    graphs, arrivals = W.serving_jobs(5, seed=7, n_hi=20000)
    assert len(graphs) == 5 and arrivals[0] == 0.0 and np.all(np.diff(arrivals) >= 0)
