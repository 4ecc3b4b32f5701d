"""Seeded synthetic graph workloads shaped like the paper's datasets.

The paper evaluates on SNAP edge lists (Eu-core, DBLP, LiveJournal,
Friendster; Datasets section, Table "Dataset Size Overview").  None of them is
shipped here, so these generators stand in for them with the same kind of
input: an undirected, unweighted edge list, possibly with duplicates and
self-loops (the Preprocessing section removes both), over non-consecutive node
ids (the "Dense Node Labels" step relabels them).

This module holds no part of the community-detection method.  It only draws
random numbers and turns them into edge lists; both the CUDA path and the CPU
oracle consume what it returns.  Every draw comes from a counter-based
splitmix64 stream (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), written out below with numpy uint64 arithmetic, so
the same seed gives the same graph on any machine and numpy version.

Workloads:

* ``planted_er``   -- 1,000 nodes, 20 planted overlapping communities of sizes
  20-150, each node in 1-3 of them, intra-community edge probability 0.15,
  Erdos-Renyi background = 2% of all edges (Eu-core stand-in).
* ``planted_chung_lu`` -- Chung-Lu power-law graph with planted overlapping
  communities of power-law sizes; used for the 335k-node (DBLP stand-in) and
  the 3.07M-node (LiveJournal/Friendster stand-in) workloads.
* small special graphs for tests (cliques, stars, cycles, paths, random).
"""
from __future__ import annotations

import dataclasses

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based splitmix64 stream: draw i is mix64(key + (i+1)*golden)."""

    def __init__(self, seed: int, stream: int):
        with np.errstate(over="ignore"):
            k = _mix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
                       + np.uint64(stream & 0xFFFFFFFF) * _GOLDEN)
        self._key = k[0]
        self._pos = 0

    def u64(self, count: int) -> np.ndarray:
        ctr = np.arange(self._pos + 1, self._pos + 1 + count, dtype=np.uint64)
        self._pos += count
        with np.errstate(over="ignore"):
            return _mix64(self._key + ctr * _GOLDEN)

    def uniform(self, count: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Integers in [lo, hi) (hi - lo < 2**32), by the multiply-shift map."""
        span = np.uint64(hi - lo)
        x = self.u64(count) >> np.uint64(32)
        with np.errstate(over="ignore"):
            return (lo + ((x * span) >> np.uint64(32)).astype(np.int64)).astype(np.int64)

    def permutation(self, count: int) -> np.ndarray:
        return np.argsort(self.u64(count), kind="stable")


@dataclasses.dataclass
class EdgeList:
    """An undirected edge list as two int32 arrays, plus generator metadata."""
    src: np.ndarray
    dst: np.ndarray
    name: str
    planted: list | None = None     # planted cover: list of int64 arrays of node ids
    params: dict | None = None

    @property
    def num_edges(self) -> int:
        return int(self.src.shape[0])


def _relabel_ids(stream: Stream, n: int, sparse: bool) -> np.ndarray:
    """Map generator node index -> external id; sparse ids leave gaps."""
    if not sparse:
        return np.arange(n, dtype=np.int64)
    gaps = stream.integers(1, 4, n)
    return np.cumsum(gaps) + 7


def planted_er(n: int = 1000, num_comms: int = 20, size_lo: int = 20, size_hi: int = 150,
               r_max: int = 3, p_in: float = 0.15, bg_frac: float = 0.02, seed: int = 0,
               sparse_ids: bool = True) -> EdgeList:
    """Planted overlapping communities with Bernoulli(p_in) inside, ER background.

    Sizes are drawn uniformly in [size_lo, size_hi], then rescaled so that they
    sum to sum_v r_v where each node's membership count r_v ~ U{1..r_max}.
    Members are dealt from a shuffled list of membership slots; a slot whose
    node already sits in the community being filled is rejected (dropped).
    """
    s = Stream(seed, 1)
    r = 1 + s.integers(0, r_max, n)
    total = int(r.sum())
    raw = s.integers(size_lo, size_hi + 1, num_comms).astype(np.float64)
    sizes = np.floor(raw * total / raw.sum()).astype(np.int64)
    sizes[np.argmax(sizes)] += total - int(sizes.sum())
    slots = np.repeat(np.arange(n, dtype=np.int64), r)
    slots = slots[s.permutation(slots.shape[0])]
    comms = []
    start = 0
    for c in range(num_comms):
        members = np.unique(slots[start:start + sizes[c]])
        start += sizes[c]
        comms.append(members)
    src_l, dst_l = [], []
    for members in comms:
        k = members.shape[0]
        iu, ju = np.triu_indices(k, 1)
        keep = s.uniform(iu.shape[0]) < p_in
        src_l.append(members[iu[keep]])
        dst_l.append(members[ju[keep]])
    intra = int(sum(a.shape[0] for a in src_l))
    n_bg = int(round(bg_frac / (1.0 - bg_frac) * intra))
    a = s.integers(0, n, n_bg)
    b = s.integers(0, n - 1, n_bg)
    b = np.where(b >= a, b + 1, b)  # no self-loops in the background draw
    src_l.append(a)
    dst_l.append(b)
    src = np.concatenate(src_l)
    dst = np.concatenate(dst_l)
    perm = s.permutation(src.shape[0])
    ids = _relabel_ids(Stream(seed, 2), n, sparse_ids)
    planted = [ids[m] for m in comms]
    return EdgeList(ids[src[perm]].astype(np.int32), ids[dst[perm]].astype(np.int32),
                    f"planted_er_n{n}_s{seed}", planted,
                    dict(n=n, num_comms=num_comms, p_in=p_in, bg_frac=bg_frac, seed=seed))


def _powerlaw_sizes(s: Stream, lo: int, hi: int, tau: float, total: int) -> np.ndarray:
    """Community sizes from a discrete power law P(s) ~ s^-tau on [lo, hi],
    drawn until they cover ``total`` membership slots."""
    est = max(16, int(2 * total / max(lo, 1)))
    while True:
        u = s.uniform(est)
        a, b = float(lo), float(hi) + 1.0
        if abs(tau - 1.0) < 1e-12:
            x = a * (b / a) ** u
        else:
            e = 1.0 - tau
            x = (a ** e + u * (b ** e - a ** e)) ** (1.0 / e)
        sizes = np.minimum(np.floor(x).astype(np.int64), hi)
        cs = np.cumsum(sizes)
        if cs[-1] >= total:
            k = int(np.searchsorted(cs, total)) + 1
            sizes = sizes[:k].copy()
            sizes[-1] -= int(cs[k - 1]) - total
            if sizes[-1] < lo:
                sizes = sizes[:-1]
                sizes[-1] += total - int(sizes.sum())
            return sizes
        est *= 2


def planted_chung_lu(n: int, avg_degree: float, gamma: float, max_degree: float,
                     size_lo: int, size_hi: int, seed: int, tau: float = 2.0,
                     r_probs=(0.55, 0.25, 0.13, 0.07), mu: float = 0.3,
                     sparse_ids: bool = True, name: str = "planted_chung_lu",
                     max_fill: float | None = None) -> EdgeList:
    """Chung-Lu power-law graph with planted overlapping communities.

    Node weights w_i ~ (i + 1)^(-1/(gamma-1)), scaled to mean ``avg_degree``
    and capped at ``max_degree``, assigned to nodes in a random order.  Each
    node joins r_v communities (r_v drawn from ``r_probs`` over 1..len) whose
    sizes follow a power law with exponent ``tau`` on [size_lo, size_hi].  A
    fraction 1-mu of the edge endpoints is drawn inside communities, each
    endpoint with probability proportional to w_v / r_v among the
    community's members (at most ``max_fill`` x its pairs, if given); the
    remaining fraction mu is a global Chung-Lu background.  Duplicate edges and self-loops are left in; the method's
    preprocessing removes them.
    """
    s = Stream(seed, 11)
    base = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    w = base * (avg_degree / base.mean())
    for _ in range(30):  # keep the mean after capping
        w = np.minimum(w, max_degree)
        w *= avg_degree / w.mean()
    w = np.minimum(w, max_degree)
    w = w[s.permutation(n)]
    cprob = np.cumsum(np.asarray(r_probs, dtype=np.float64))
    cprob /= cprob[-1]
    r = 1 + np.searchsorted(cprob, s.uniform(n), side="right").astype(np.int64)
    r = np.minimum(r, len(r_probs))
    total = int(r.sum())
    sizes = _powerlaw_sizes(s, size_lo, size_hi, tau, total)
    slots = np.repeat(np.arange(n, dtype=np.int64), r)
    slots = slots[s.permutation(slots.shape[0])]
    comm_of_slot = np.repeat(np.arange(sizes.shape[0], dtype=np.int64), sizes)
    # duplicate rejection: a node dealt twice into one community keeps one slot
    key = comm_of_slot * n + slots
    key = np.unique(key)
    m_comm = key // n
    m_node = key % n
    num_comms = int(sizes.shape[0])
    # per-membership intra weight a_{v,c} = w_v / r_v, grouped by community
    a = w[m_node] / r[m_node]
    cum = np.cumsum(a)
    starts = np.searchsorted(m_comm, np.arange(num_comms), side="left")
    ends = np.searchsorted(m_comm, np.arange(num_comms), side="right")
    cum0 = np.concatenate([[0.0], cum])
    A = cum0[ends] - cum0[starts]
    target_edges = n * avg_degree / 2.0
    e_intra = (1.0 - mu) * target_edges * A / A.sum()
    # integer edge budgets with a random rounding
    e_c = np.floor(e_intra + s.uniform(num_comms)).astype(np.int64)
    sz = (ends - starts).astype(np.int64)
    if max_fill is not None:   # keep small communities from saturating (their draws would repeat)
        e_c = np.minimum(e_c, np.floor(max_fill * sz * (sz - 1) / 2.0).astype(np.int64))
    e_c = np.where(sz >= 2, e_c, 0)
    n_in = int(e_c.sum())
    comm_of_edge = np.repeat(np.arange(num_comms, dtype=np.int64), e_c)

    def draw_in(count_per_edge_comm):
        lo = cum0[starts[count_per_edge_comm]]
        hi = cum0[ends[count_per_edge_comm]]
        u = lo + s.uniform(count_per_edge_comm.shape[0]) * (hi - lo)
        idx = np.searchsorted(cum, u, side="right")
        idx = np.clip(idx, starts[count_per_edge_comm], ends[count_per_edge_comm] - 1)
        return m_node[idx]

    src_in = draw_in(comm_of_edge)
    dst_in = draw_in(comm_of_edge)
    n_bg = int(round(mu * target_edges))
    gcum = np.cumsum(w)
    src_bg = np.searchsorted(gcum, s.uniform(n_bg) * gcum[-1], side="right")
    dst_bg = np.searchsorted(gcum, s.uniform(n_bg) * gcum[-1], side="right")
    src_bg = np.minimum(src_bg, n - 1)
    dst_bg = np.minimum(dst_bg, n - 1)
    src = np.concatenate([src_in, src_bg])
    dst = np.concatenate([dst_in, dst_bg])
    # every node appears: a node that drew no non-loop edge gets one background edge
    touched = np.zeros(n, dtype=bool)
    nl = src != dst
    touched[src[nl]] = True
    touched[dst[nl]] = True
    lonely = np.flatnonzero(~touched)
    if lonely.shape[0]:
        partner = np.searchsorted(gcum, s.uniform(lonely.shape[0]) * gcum[-1], side="right")
        partner = np.minimum(partner, n - 1)
        partner = np.where(partner == lonely, (partner + 1) % n, partner)
        src = np.concatenate([src, lonely])
        dst = np.concatenate([dst, partner])
    ids = _relabel_ids(Stream(seed, 12), n, sparse_ids)
    if ids[-1] >= 2**31:
        raise ValueError("external ids exceed int32")
    planted = None
    if n <= 400_000:
        order = np.argsort(m_comm, kind="stable")
        planted = np.split(ids[m_node[order]], np.cumsum(np.bincount(m_comm, minlength=num_comms))[:-1])
    return EdgeList(ids[src].astype(np.int32), ids[dst].astype(np.int32),
                    f"{name}_n{n}_s{seed}", planted,
                    dict(n=n, avg_degree=avg_degree, gamma=gamma, max_degree=max_degree,
                         size_lo=size_lo, size_hi=size_hi, tau=tau, mu=mu, seed=seed,
                         intra_edges=n_in, background_edges=n_bg))


# --- the named workloads ----------------------------------------------------

def eu_core_like(seed: int = 0) -> EdgeList:
    """1,000 nodes, 20 planted communities (sizes 20-150, 1-3 per node),
    p_in 0.15, 2% ER background; Fox (queue size 1), threshold 0.01, 50 iters."""
    return planted_er(1000, 20, 20, 150, 3, 0.15, 0.02, seed)


def dblp_like(seed: int = 1, scale: float = 1.0) -> EdgeList:
    """335k nodes, ~0.93M edges, degree exponent 2.5, max degree ~550,
    planted community sizes 6-2,000, each node in 1-4 (queue sizes 64, 1024).
    ``scale`` < 1 gives a proportionally smaller graph for quick tests."""
    n = max(200, int(round(335_000 * scale)))
    return planted_chung_lu(n, avg_degree=6.45, gamma=2.5, max_degree=700.0,
                            size_lo=6, size_hi=2000, seed=seed, name="dblp_like")


def large_like(seed: int = 4, scale: float = 1.0) -> EdgeList:
    """3.07M nodes, ~117M edges, degree exponent 2.2, max degree ~33k,
    planted community sizes 10-5,000 (queue sizes 1024, 65536; 20 iterations)."""
    n = max(1000, int(round(3_070_000 * scale)))
    # weight cap above the target maximum degree: a hub's weight is split over
    # saturated communities and the background, realising ~32k neighbours
    return planted_chung_lu(n, avg_degree=136.0, gamma=2.2, max_degree=95_000.0,
                            size_lo=10, size_hi=5000, seed=seed, name="large_like", max_fill=0.5)


# --- small graphs for tests ---------------------------------------------------

def from_pairs(pairs, name="pairs") -> EdgeList:
    arr = np.asarray(list(pairs), dtype=np.int64).reshape(-1, 2)
    return EdgeList(arr[:, 0].astype(np.int32), arr[:, 1].astype(np.int32), name)


def clique(k: int, offset: int = 0):
    return [(offset + i, offset + j) for i in range(k) for j in range(i + 1, k)]


def star(k: int, center: int = 0):
    return [(center, center + 1 + i) for i in range(k)]


def cycle(k: int, offset: int = 0):
    return [(offset + i, offset + (i + 1) % k) for i in range(k)]


def path(k: int, offset: int = 0):
    return [(offset + i, offset + i + 1) for i in range(k - 1)]


def random_graph(n: int, m: int, seed: int, hubs: int = 0, hub_degree: int = 0,
                 self_loops: int = 0, duplicates: int = 0) -> EdgeList:
    """Uniform random pairs, optionally with a few high-degree hubs, self-loops
    and repeated pairs (to exercise every preprocessing branch)."""
    s = Stream(seed, 21)
    a = s.integers(0, n, m)
    b = s.integers(0, n, m)
    parts_a, parts_b = [a], [b]
    for h in range(hubs):
        nb = s.integers(0, n, hub_degree)
        parts_a.append(np.full(hub_degree, h * 7 % n, dtype=np.int64))
        parts_b.append(nb)
    if self_loops:
        v = s.integers(0, n, self_loops)
        parts_a.append(v)
        parts_b.append(v)
    src = np.concatenate(parts_a)
    dst = np.concatenate(parts_b)
    if duplicates:
        pick = s.integers(0, src.shape[0], duplicates)
        src = np.concatenate([src, dst[pick]])
        dst = np.concatenate([dst, src[pick]])
    return EdgeList(src.astype(np.int32), dst.astype(np.int32), f"random_n{n}_m{m}_s{seed}")


def wide_fan(spokes: int = 2100, leaves: int = 20000, leaf_degree: int = 252, chords: int = 5000,
             seed: int = 0) -> EdgeList:
    """A centre joined to `spokes` nodes that are busier than it (each leaf
    picks `leaf_degree` random spokes, plus `chords` random spoke-spoke
    edges), so that the degree orientation gives the centre an out-degree of
    about `spokes` and every leaf one of `leaf_degree`: the out-degree range
    that per-warp triangle work cannot hold."""
    s = Stream(seed, 23)
    centre = np.zeros(spokes, np.int64)
    sp = np.arange(1, spokes + 1, dtype=np.int64)
    leaf = np.repeat(np.arange(spokes + 1, spokes + 1 + leaves, dtype=np.int64), leaf_degree)
    pick = 1 + s.integers(0, spokes, leaves * leaf_degree)
    ca = 1 + s.integers(0, spokes, chords)
    cb = 1 + s.integers(0, spokes, chords)
    src = np.concatenate([centre, leaf, ca])
    dst = np.concatenate([sp, pick, cb])
    return EdgeList(src.astype(np.int32), dst.astype(np.int32), f"wide_fan_{spokes}_{leaves}x{leaf_degree}")


def hub_of_triangles(triangles: int = 10000, extra: int = 2, hub_links: int = 2, seed: int = 0) -> EdgeList:
    """A hub joined to `hub_links` corners of each of `triangles` disjoint
    triangles (and, from each first corner, to `extra` random other first
    corners), so that the hub's neighbours bring one distinct community per
    triangle: a hub with more candidate communities than one block evaluates
    at once."""
    s = Stream(seed, 29)
    t = np.arange(triangles, dtype=np.int64)
    a, b, c = 1 + 3 * t, 2 + 3 * t, 3 + 3 * t
    zero = np.zeros(triangles, np.int64)
    src = [a, b, a, zero] + ([zero] if hub_links > 1 else [])
    dst = [b, c, c, a] + ([b] if hub_links > 1 else [])
    if extra:
        src.append(np.repeat(a, extra))
        dst.append(1 + 3 * s.integers(0, triangles, triangles * extra))
    return EdgeList(np.concatenate(src).astype(np.int32), np.concatenate(dst).astype(np.int32),
                    f"hub_of_{triangles}_triangles")


def batched_planted(count: int = 4096, seed: int = 5, n_lo: int = 200, n_hi: int = 20000,
                    deg_lo: float = 8.0, deg_hi: float = 40.0) -> list:
    """The batched workload: `count` independent planted graphs with node
    counts log-uniform in [n_lo, n_hi] and average degree uniform in
    [deg_lo, deg_hi], planted overlapping communities as in `planted_er`
    (sizes 20-150, 1-3 per node, 2% background).  With 2 memberships per node
    on average and communities of ~85 nodes, p_in = degree / 170 gives the
    requested average degree."""
    s = Stream(seed, 31)
    ln = s.uniform(count) * (np.log(n_hi) - np.log(n_lo)) + np.log(n_lo)
    ns = np.maximum(n_lo, np.round(np.exp(ln))).astype(np.int64)
    degs = deg_lo + s.uniform(count) * (deg_hi - deg_lo)
    out = []
    for i in range(count):
        n = int(ns[i])
        out.append(planted_er(n=n, num_comms=max(2, int(round(2 * n / 85))), p_in=min(1.0, float(degs[i]) / 170.0),
                              seed=seed * 100003 + i))
    return out


def serving_jobs(count: int = 64, seed: int = 7, n_lo: int = 1000, n_hi: int = 2_000_000, deg_lo: float = 10.0,
                 deg_hi: float = 80.0, rate: float = 200.0) -> tuple:
    """The serving workload: `count` planted graphs with node counts
    log-uniform in [n_lo, n_hi] and average degree uniform in [deg_lo,
    deg_hi] (as `batched_planted`), arriving as a Poisson stream of `rate`
    jobs per second.  Returns (graphs, arrival times in seconds from 0)."""
    s = Stream(seed, 37)
    ln = s.uniform(count) * (np.log(n_hi) - np.log(n_lo)) + np.log(n_lo)
    ns = np.maximum(n_lo, np.round(np.exp(ln))).astype(np.int64)
    degs = deg_lo + s.uniform(count) * (deg_hi - deg_lo)
    gaps = -np.log(1.0 - s.uniform(count)) / rate
    arrivals = np.cumsum(gaps) - gaps[0]
    graphs = [planted_er(n=int(ns[i]), num_comms=max(2, int(round(2 * ns[i] / 85))),
                         p_in=min(1.0, float(degs[i]) / 170.0), seed=seed * 100019 + i) for i in range(count)]
    return graphs, arrivals
