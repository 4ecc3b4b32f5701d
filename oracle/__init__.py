"""ctypes wrapper of the sequential CPU oracle (``lazyfox_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never loads it
and shares no code with it.  ``build()`` compiles the C file with gcc
(``-O2 -ffp-contract=off``: no fused multiply-add, so every FP64 expression is
rounded operation by operation as written).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lazyfox_oracle.c")
_LIB = os.path.join(_HERE, "liblazyfox_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_P = C.c_void_p
_I64P = C.POINTER(C.c_int64)
_I32P = C.POINTER(C.c_int32)
_F64P = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        sig = {
            "og_create": (_P, [_I32P, _I32P, C.c_int64, C.POINTER(C.c_int)]),
            "og_destroy": (None, [_P]),
            "og_prepare": (C.c_int, [_P]),
            "og_triangles": (C.c_int, [_P]),
            "og_order": (C.c_int, [_P]),
            "og_sizes": (None, [_P, _I64P, _I64P]),
            "og_get_csr": (None, [_P, _I64P, _I32P, _I32P]),
            "og_get_node_stats": (C.c_int, [_P, _I64P, _I32P, _F64P]),
            "og_get_order": (C.c_int, [_P, _I32P]),
            "og_node_triangles": (C.c_int64, [_P, C.c_int32, _I32P]),
            "og_local_cc": (C.c_double, [_P, C.c_int64]),
            "og_init_clustering": (C.c_int, [_P]),
            "og_run": (C.c_int, [_P, C.c_int32, C.c_double, C.c_int32, C.c_int64]),
            "og_num_comm_ids": (C.c_int64, [_P]),
            "og_num_memberships": (C.c_int64, [_P]),
            "og_get_state": (None, [_P, _I64P, _I32P, _I64P, _I64P, _I64P]),
            "og_get_run": (None, [_P, _I32P, _I32P, _F64P, _F64P, _I64P, _I64P, C.c_int32]),
            "og_set_check_invariants": (None, [_P, C.c_int]),
            "og_set_partition": (C.c_int, [_P, _I64P, _I32P, C.c_int64]),
            "og_f1_pair": (C.c_double, [C.c_int64, C.c_int64, C.c_int64]),
            "og_cover_f1": (C.c_int, [_I64P, _I32P, C.c_int64, _I64P, _I32P, C.c_int64, _F64P, _I32P]),
            "og_invariant_failures": (C.c_int, [_P]),
            "og_evaluate": (None, [_P, C.c_int32, _I32P, _I32P, _I64P, _I64P, _F64P, _F64P]),
            "og_total": (C.c_double, [_P]),
            "og_total_meanfield": (C.c_double, [_P]),
            "og_get_cc": (C.c_double, [_P]),
            "og_fsum": (C.c_double, [_F64P, C.c_int64]),
            "og_wcchat_node": (C.c_double, [C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_double]),
            "og_community_score": (C.c_double, [C.c_int64, C.c_int64, C.c_int64, C.c_double]),
            "og_exact_wcc": (C.c_double, [_P, C.c_int32, _I32P, C.c_int64]),
            "og_adjacent": (C.c_int, [_P, C.c_int32, C.c_int32]),
            "og_literal_gain": (C.c_double, [_P, C.c_int32, C.c_int32]),
            "og_evaluate_literal": (None, [_P, C.c_int32, _I32P, _I32P, _F64P, _F64P]),
            "og_set_literal_diagnostic": (None, [_P, C.c_int]),
            "og_get_literal_diagnostic": (None, [_P, _I64P]),
            "og_get_meanfield_history": (None, [_P, _F64P, C.c_int32]),
            "og_set_gain_rule": (C.c_int, [_P, C.c_int]),
            "og_get_gain_rule": (C.c_int, [_P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def fsum(values) -> float:
    a = np.ascontiguousarray(values, dtype=np.float64)
    return lib().og_fsum(_ptr(a, C.c_double), a.shape[0])


def wcchat_node(k, d, n, m, cc) -> float:
    return lib().og_wcchat_node(int(k), int(d), int(n), int(m), float(cc))


def community_score(n, m, vol, cc) -> float:
    return lib().og_community_score(int(n), int(m), int(vol), float(cc))


def _cover_csr(cover):
    sizes = np.array([len(c) for c in cover], dtype=np.int64)
    off = np.zeros(len(cover) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    mem = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int32) for c in cover])
                               if len(cover) and off[-1] > 0 else np.zeros(1, dtype=np.int32))
    return off, mem


def cover_f1(detected, reference):
    """F1-score of a detected cover against a reference cover (lists of id
    arrays) and, per detected community, the index of its best reference
    community (-1 if it shares no node with any)."""
    oa, ma = _cover_csr(detected)
    ob, mb = _cover_csr(reference)
    f1 = C.c_double()
    best = np.zeros(max(1, len(detected)), dtype=np.int32)
    lib().og_cover_f1(_ptr(oa, C.c_int64), _ptr(ma, C.c_int32), len(detected), _ptr(ob, C.c_int64),
                      _ptr(mb, C.c_int32), len(reference), C.byref(f1), _ptr(best, C.c_int32))
    return f1.value, best[:len(detected)]


def f1_pair(k: int, a: int, b: int) -> float:
    return lib().og_f1_pair(int(k), int(a), int(b))


def _run_one(job):
    src, dst, q, threshold, max_iters, rule = job
    g = OracleGraph(src, dst)
    r = g.run(q, threshold, max_iters, rule=rule)
    r["cc"] = g.cc
    r["communities"] = [c.tolist() for c in g.communities()]
    return r


def run_many(edge_lists, queue_size, threshold, max_iters, rule=None, processes=None):
    """Independent oracle runs of many graphs (objects with src/dst), one
    spawned process per host core (largest graphs first); per graph the run's
    record with its cc and final communities (lists of original ids), in the
    order of `edge_lists`."""
    import multiprocessing as mp
    jobs = [(el.src, el.dst, queue_size, threshold, max_iters, rule) for el in edge_lists]
    procs = min(len(jobs), processes or len(os.sched_getaffinity(0)))
    if procs <= 1:
        return [_run_one(j) for j in jobs]
    order = sorted(range(len(jobs)), key=lambda i: -jobs[i][0].shape[0])
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_run_one, [jobs[i] for i in order], chunksize=1)
    out = [None] * len(jobs)
    for i, r in zip(order, res):
        out[i] = r
    return out


class OracleGraph:
    """The oracle's view of one graph: preprocessing, triangles, order, runs."""

    def __init__(self, src, dst, prepare: bool = True):
        L = lib()
        self._src = np.ascontiguousarray(src, dtype=np.int32)
        self._dst = np.ascontiguousarray(dst, dtype=np.int32)
        st = C.c_int(0)
        self._h = L.og_create(_ptr(self._src, C.c_int32), _ptr(self._dst, C.c_int32),
                              self._src.shape[0], C.byref(st))
        if not self._h:
            raise ValueError(f"oracle rejected the edge list (status {st.value})")
        n, m = C.c_int64(), C.c_int64()
        L.og_sizes(self._h, C.byref(n), C.byref(m))
        self.n, self.m = n.value, m.value
        if prepare:
            self.prepare()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().og_destroy(h)
            self._h = None

    def prepare(self):
        st = lib().og_prepare(self._h)
        if st:
            raise RuntimeError(f"og_prepare failed {st}")

    def csr(self):
        off = np.empty(self.n + 1, dtype=np.int64)
        adj = np.empty(max(1, 2 * self.m), dtype=np.int32)
        labels = np.empty(max(1, self.n), dtype=np.int32)
        lib().og_get_csr(self._h, _ptr(off, C.c_int64), _ptr(adj, C.c_int32), _ptr(labels, C.c_int32))
        return off, adj[:2 * self.m], labels[:self.n]

    def node_stats(self):
        t = np.empty(max(1, self.n), dtype=np.int64)
        vt = np.empty(max(1, self.n), dtype=np.int32)
        cc = C.c_double()
        st = lib().og_get_node_stats(self._h, _ptr(t, C.c_int64), _ptr(vt, C.c_int32), C.byref(cc))
        if st:
            raise RuntimeError("triangles not computed")
        return t[:self.n], vt[:self.n], cc.value

    def node_triangles(self, x: int):
        vt = C.c_int32()
        t = lib().og_node_triangles(self._h, int(x), C.byref(vt))
        return t, vt.value

    def order(self):
        o = np.empty(max(1, self.n), dtype=np.int32)
        if lib().og_get_order(self._h, _ptr(o, C.c_int32)):
            raise RuntimeError("order not computed")
        return o[:self.n]

    def local_cc(self, x: int) -> float:
        return lib().og_local_cc(self._h, int(x))

    @property
    def cc(self) -> float:
        return lib().og_get_cc(self._h)

    def init_clustering(self):
        if lib().og_init_clustering(self._h):
            raise RuntimeError("order not computed")

    def set_partition(self, communities):
        """Insert a division (list of arrays of original ids) that replaces the
        initial clustering of the following runs; None removes it."""
        if communities is None:
            lib().og_set_partition(self._h, None, None, -1)
            return
        sizes = np.array([len(c) for c in communities], dtype=np.int64)
        off = np.zeros(len(communities) + 1, dtype=np.int64)
        np.cumsum(sizes, out=off[1:])
        mem = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int32) for c in communities])
                                   if communities else np.zeros(1, dtype=np.int32))
        st = lib().og_set_partition(self._h, _ptr(off, C.c_int64), _ptr(mem, C.c_int32), len(communities))
        if st:
            raise ValueError(f"og_set_partition failed {st}")

    GAIN_RULES = {"literal": 0, "meanfield": 1}

    def set_gain_rule(self, rule: str):
        """Decision rule of the following runs: "literal" (the paper's gain, the
        change of \\wcchat(P); the default) or "meanfield" (the change of the
        mean-field community score, a departure kept as an option)."""
        if rule not in self.GAIN_RULES or lib().og_set_gain_rule(self._h, self.GAIN_RULES[rule]):
            raise ValueError(f"unknown gain rule {rule!r}")

    @property
    def gain_rule(self) -> str:
        v = lib().og_get_gain_rule(self._h)
        return next(k for k, c in self.GAIN_RULES.items() if c == v)

    def set_check_invariants(self, on: bool):
        lib().og_set_check_invariants(self._h, 1 if on else 0)

    def invariant_failures(self) -> int:
        return lib().og_invariant_failures(self._h)

    def run(self, queue_size: int, threshold: float, max_iters: int, max_batches: int = -1, rule=None):
        if rule is not None:
            self.set_gain_rule(rule)
        st = lib().og_run(self._h, int(queue_size), float(threshold), int(max_iters), int(max_batches))
        if st:
            raise ValueError(f"og_run failed {st}")
        return self.run_info(max(1, max_iters))

    def run_info(self, cap: int):
        it, conv, T0 = C.c_int32(), C.c_int32(), C.c_double()
        T = np.zeros(cap, dtype=np.float64)
        j = np.zeros(cap, dtype=np.int64)
        lv = np.zeros(cap, dtype=np.int64)
        lib().og_get_run(self._h, C.byref(it), C.byref(conv), C.byref(T0), _ptr(T, C.c_double),
                         _ptr(j, C.c_int64), _ptr(lv, C.c_int64), cap)
        k = it.value
        S = np.zeros(cap, dtype=np.float64)
        lib().og_get_meanfield_history(self._h, _ptr(S, C.c_double), cap)
        return dict(iterations=k, converged=bool(conv.value), T0=T0.value,
                    T=T[:k].copy(), joins=j[:k].copy(), leaves=lv[:k].copy(), S=S[:k].copy())

    def state(self):
        """Memberships (CSR over dense ids) and aggregates for every community id.

        Aggregates: members n_C, internal edges m_C, member-degree sum vol_C."""
        L = lib()
        k = L.og_num_comm_ids(self._h)
        nm = L.og_num_memberships(self._h)
        mem_off = np.empty(self.n + 1, dtype=np.int64)
        mem_ids = np.empty(max(1, nm), dtype=np.int32)
        cn = np.empty(max(1, k), dtype=np.int64)
        cm = np.empty(max(1, k), dtype=np.int64)
        cv = np.empty(max(1, k), dtype=np.int64)
        L.og_get_state(self._h, _ptr(mem_off, C.c_int64), _ptr(mem_ids, C.c_int32),
                       _ptr(cn, C.c_int64), _ptr(cm, C.c_int64), _ptr(cv, C.c_int64))
        return dict(mem_off=mem_off, mem_ids=mem_ids[:nm], n=cn[:k], m=cm[:k], vol=cv[:k])

    def evaluate(self, x: int):
        j, lv = C.c_int32(), C.c_int32()
        kj, kl = C.c_int64(), C.c_int64()
        gj, gl = C.c_double(), C.c_double()
        lib().og_evaluate(self._h, int(x), C.byref(j), C.byref(lv), C.byref(kj), C.byref(kl),
                          C.byref(gj), C.byref(gl))
        return dict(join=j.value, leave=lv.value, kjoin=kj.value, kleave=kl.value,
                    gjoin=gj.value, gleave=gl.value)

    def total(self) -> float:
        return lib().og_total(self._h)

    def literal_gain(self, x: int, c: int) -> float:
        """Change of the literal \\wcchat(P) if x alone joins c (not a member)
        or leaves it (a member); a diagnostic of the gain reading."""
        return lib().og_literal_gain(self._h, int(x), int(c))

    def evaluate_literal(self, x: int):
        """x's decision with literal gains instead of mean-field ones."""
        j, lv = C.c_int32(), C.c_int32()
        gj, gl = C.c_double(), C.c_double()
        lib().og_evaluate_literal(self._h, int(x), C.byref(j), C.byref(lv), C.byref(gj), C.byref(gl))
        return dict(join=j.value, leave=lv.value, gjoin=gj.value, gleave=gl.value)

    def set_literal_diagnostic(self, on: bool):
        """Following runs also take every decision with literal gains and count agreement."""
        lib().og_set_literal_diagnostic(self._h, 1 if on else 0)

    def literal_diagnostic(self) -> dict:
        out = np.zeros(8, dtype=np.int64)
        lib().og_get_literal_diagnostic(self._h, _ptr(out, C.c_int64))
        keys = ("evaluations", "same_join", "same_leave", "same_both", "joins_meanfield", "joins_literal",
                "leaves_meanfield", "leaves_literal")
        return {k: int(v) for k, v in zip(keys, out)}

    def total_meanfield(self) -> float:
        return lib().og_total_meanfield(self._h)

    def exact_wcc(self, x: int, members) -> float:
        mm = np.ascontiguousarray(np.sort(np.asarray(members, dtype=np.int32)))
        return lib().og_exact_wcc(self._h, int(x), _ptr(mm, C.c_int32), mm.shape[0])

    def adjacent(self, x: int, y: int) -> bool:
        return bool(lib().og_adjacent(self._h, int(x), int(y)))

    def communities(self):
        """Live communities, ascending id, members ascending, original labels."""
        s = self.state()
        _, _, labels = self.csr()
        live = np.flatnonzero(s["n"] > 0)
        out = {int(c): [] for c in live}
        for x in range(self.n):
            for c in s["mem_ids"][s["mem_off"][x]:s["mem_off"][x + 1]]:
                out[int(c)].append(int(labels[x]))
        return [np.asarray(out[int(c)], dtype=np.int32) for c in live]
