"""Python binding of the LazyFox C ABI (``include/lazyfox.h``).

Argument marshalling only: every step of the method runs in the CUDA library
``lib/liblazyfox.so``.  PyTorch supplies the device memory (its caching
allocator, through the ABI's allocation callbacks) and the CUDA stream.  There
is no fallback: if the library or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "liblazyfox.so")

LF_OK, LF_ERR_INVALID, LF_ERR_OOM, LF_ERR_CUDA, LF_ERR_CAPACITY, LF_ERR_TIMEOUT, LF_ERR_STATE = range(7)
_STATUS = {1: "LF_ERR_INVALID", 2: "LF_ERR_OOM", 3: "LF_ERR_CUDA", 4: "LF_ERR_CAPACITY",
           5: "LF_ERR_TIMEOUT", 6: "LF_ERR_STATE"}

ABI_FUNCTIONS = ("lf_graph_create", "lf_run", "lf_run_partial", "lf_get_communities",
                 "lf_get_node_stats", "lf_get_sizes", "lf_get_create_stats", "lf_get_csr",
                 "lf_get_oriented", "lf_get_order", "lf_get_state", "lf_graph_destroy",
                 "lf_last_error", "lf_triangles_noalloc", "lf_set_partition", "lf_set_iteration_callback",
                 "lf_batch_create", "lf_batch_get_info", "lf_batch_get_history", "lf_batch_get_communities",
                 "lf_autotune", "lf_server_create", "lf_server_submit", "lf_server_wait",
                 "lf_server_get_communities", "lf_server_release", "lf_server_destroy", "lf_cover_f1")


# lf_options.gain_rule: None = the library default; "literal" = the paper's gain
# (the change of WCC-hat(P)); "meanfield" = the mean-field departure
GAIN_RULES = {None: 0, "literal": 1, "meanfield": 2}


class LazyFoxError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_ITER_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int32, C.c_double, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN),
                ("alloc_ctx", C.c_void_p), ("edges_on_device", C.c_int32),
                ("member_slots", C.c_int32), ("warp_max_degree", C.c_int32),
                ("use_graphs", C.c_int32), ("profile", C.c_int32), ("exhaustive_fp64", C.c_int32),
                ("per_queue_launches", C.c_int32), ("barrier_timeout_ms", C.c_int32),
                ("inject_barrier_stall", C.c_int32), ("barrier_mode", C.c_int32),
                ("warps_per_node", C.c_int32), ("hub_degree", C.c_int32), ("gain_rule", C.c_int32),
                ("debug_checks", C.c_int32)]


class RunStatsC(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("num_batches", C.c_int64),
                ("wcc_initial", C.c_double), ("num_communities", C.c_int64),
                ("num_memberships", C.c_int64), ("ms_total", C.c_double), ("ms_init", C.c_double),
                ("ms_iterations", C.c_double), ("history_cap", C.c_int32),
                ("wcc_history", C.POINTER(C.c_double)), ("joins_history", C.POINTER(C.c_int64)),
                ("leaves_history", C.POINTER(C.c_int64)), ("num_launches", C.c_int64),
                ("prof_move_launches", C.c_int64), ("prof_move_ms", C.c_double),
                ("prof_move_bytes", C.c_int64), ("prof_queue_us", C.c_double * 4),
                ("prof_candidates", C.c_int64), ("prof_exact", C.c_int64)]


class TuneResultC(C.Structure):
    _fields_ = [("warps_per_node", C.c_int32), ("warp_max_degree", C.c_int32), ("trials", C.c_int32),
                ("hub_degree", C.c_int32), ("best_ms", C.c_double), ("default_ms", C.c_double)]


class ServerOptionsC(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_active", C.c_int32), ("pad", C.c_int32)]


class JobResultC(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("converged", C.c_int32), ("pad", C.c_int32),
                ("wcc_initial", C.c_double), ("wcc_final", C.c_double), ("num_nodes", C.c_int64),
                ("num_edges", C.c_int64), ("num_communities", C.c_int64), ("est_bytes", C.c_int64),
                ("t_submit_ms", C.c_double), ("t_admit_ms", C.c_double), ("t_done_ms", C.c_double)]


class CreateStatsC(C.Structure):
    _fields_ = [("num_nodes", C.c_int64), ("num_edges", C.c_int64), ("num_triangles", C.c_int64),
                ("ms_csr", C.c_double), ("ms_orient", C.c_double), ("ms_triangles", C.c_double),
                ("ms_vt", C.c_double), ("ms_order", C.c_double), ("merge_bytes", C.c_int64),
                ("num_launches", C.c_int64)]


_lib = None


def load_library(path: str | None = None) -> C.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise LazyFoxError(LF_ERR_STATE, f"CUDA library not built: {p} (run paper_2210_03211_gb300.build)")
    L = C.CDLL(p)
    P = C.c_void_p
    i64p, i32p, f64p = C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double)
    sig = {
        "lf_graph_create": (C.c_int, [P, P, C.c_int64, C.POINTER(Options), C.POINTER(P)]),
        "lf_run": (C.c_int, [P, C.c_int32, C.c_double, C.c_int32, C.POINTER(RunStatsC)]),
        "lf_run_partial": (C.c_int, [P, C.c_int32, C.c_double, C.c_int32, C.c_int64, C.POINTER(RunStatsC)]),
        "lf_get_communities": (C.c_int, [P, i64p, C.c_int64, i32p, C.c_int64, i64p, i64p]),
        "lf_get_node_stats": (C.c_int, [P, i64p, i32p, f64p]),
        "lf_get_sizes": (C.c_int, [P, i64p, i64p]),
        "lf_get_create_stats": (C.c_int, [P, C.POINTER(CreateStatsC)]),
        "lf_get_csr": (C.c_int, [P, i64p, i32p, i32p]),
        "lf_get_oriented": (C.c_int, [P, i64p, i32p]),
        "lf_get_order": (C.c_int, [P, i32p]),
        "lf_get_state": (C.c_int, [P, i64p, i32p, i64p, i64p, i64p, i64p, i64p]),
        "lf_graph_destroy": (None, [P]),
        "lf_last_error": (C.c_char_p, []),
        "lf_triangles_noalloc": (C.c_int, [P, P, C.c_int64, C.c_int64, P, P, P]),
        "lf_set_partition": (C.c_int, [P, i64p, i32p, C.c_int64]),
        "lf_set_iteration_callback": (C.c_int, [P, _ITER_FN, P]),
        "lf_batch_create": (C.c_int, [P, P, i64p, C.c_int64, C.POINTER(Options), C.POINTER(P)]),
        "lf_batch_get_info": (C.c_int, [P, i64p, i64p, i32p, i32p, f64p, f64p, f64p]),
        "lf_batch_get_history": (C.c_int, [P, C.c_int64, f64p, C.c_int32, i32p]),
        "lf_batch_get_communities": (C.c_int, [P, i64p, i64p, C.c_int64, i32p, C.c_int64, i64p, i64p]),
        "lf_autotune": (C.c_int, [P, C.c_int32, C.c_int32, C.POINTER(TuneResultC)]),
        "lf_server_create": (C.c_int, [C.POINTER(ServerOptionsC), C.POINTER(P)]),
        "lf_server_submit": (C.c_int, [P, P, P, C.c_int64, C.c_int32, C.c_double, C.c_int32, i64p]),
        "lf_server_wait": (C.c_int, [P, C.c_int64, C.c_double, C.POINTER(JobResultC)]),
        "lf_server_get_communities": (C.c_int, [P, C.c_int64, i64p, C.c_int64, i32p, C.c_int64, i64p, i64p]),
        "lf_server_release": (C.c_int, [P, C.c_int64]),
        "lf_server_destroy": (None, [P]),
        "lf_cover_f1": (C.c_int, [i64p, i32p, C.c_int64, i64p, i32p, C.c_int64, f64p, i32p, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = L
    return L


def _check(L, status: int):
    if status != LF_OK:
        raise LazyFoxError(status, L.lf_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self._device = device
        self.alloc = _ALLOC_FN(self._alloc)
        self.free = _FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), self._device, stream)
        except Exception:  # noqa: BLE001 - an allocation failure is reported to the library as NULL
            return None

    def _free(self, ptr, nbytes, stream, ctx):
        if ptr:
            self._torch.cuda.caching_allocator_delete(ptr)


class CountingAllocator(_TorchAllocator):
    """The torch allocator bridge with accounting: allocations made, bytes live
    and their peak.  ``fail_at`` (1-based) makes that allocation return NULL,
    as a failing device allocator would (the library then reports
    LF_ERR_OOM).  Pass it as ``Graph(..., allocator=CountingAllocator(dev))``."""

    def __init__(self, device, fail_at=None):
        super().__init__(device)
        self.fail_at = fail_at
        self.calls = 0
        self.live = 0
        self.peak = 0
        self._sizes = {}

    def _alloc(self, nbytes, stream, ctx):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return None
        ptr = super()._alloc(nbytes, stream, ctx)
        if ptr:
            self._sizes[ptr] = int(nbytes)
            self.live += int(nbytes)
            self.peak = max(self.peak, self.live)
        return ptr

    def _free(self, ptr, nbytes, stream, ctx):
        if ptr:
            self.live -= self._sizes.pop(ptr, 0)
        super()._free(ptr, nbytes, stream, ctx)


@dataclasses.dataclass
class RunStats:
    iterations: int
    converged: bool
    num_batches: int
    wcc_initial: float
    wcc_history: np.ndarray
    joins: np.ndarray
    leaves: np.ndarray
    num_communities: int
    num_memberships: int
    ms_total: float
    ms_init: float
    ms_iterations: float
    num_launches: int = 0
    prof_move_launches: int = 0
    prof_move_ms: float = 0.0
    prof_move_bytes: int = 0
    prof_queue_us: tuple = (0.0, 0.0, 0.0, 0.0)
    prof_candidates: int = 0
    prof_exact: int = 0


class Graph:
    """One graph on the GPU: ``lf_graph_create`` plus the run and result calls.

    ``src``/``dst``: numpy int32 arrays (host) or int32 CUDA tensors (device).
    ``stream``: a ``torch.cuda.Stream`` (default: torch's current stream).
    ``allocator``: "torch" (caching allocator), "cuda" (cudaMallocAsync) or a
    :class:`CountingAllocator`.
    """

    def __init__(self, src, dst, *, stream=None, allocator: str = "torch", member_slots: int = 0,
                 warp_max_degree: int = 0, use_graphs: bool = True, profile: bool = False,
                 exhaustive_fp64: bool = False, per_queue_launches: bool | None = None,
                 barrier_timeout_ms: int = 0, inject_barrier_stall: bool = False, barrier_mode: int = 0,
                 warps_per_node: int = 0, hub_degree: int = 0, gain_rule: str | None = None,
                 debug_checks: bool = False, device=None, edge_offsets=None):
        import torch
        self._L = load_library()
        self._h = C.c_void_p()
        if not torch.cuda.is_available():
            raise LazyFoxError(LF_ERR_CUDA, "no CUDA device available")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        if stream is None:
            # a stream of our own, ordered after the caller's current stream (which
            # produced any device-resident edge list)
            stream = torch.cuda.Stream(self.device)
            stream.wait_stream(torch.cuda.current_stream(self.device))
        self.stream = stream
        opt = Options()
        opt.stream = C.c_void_p(self.stream.cuda_stream)
        self._allocator = None
        if allocator == "torch":
            self._allocator = _TorchAllocator(self.device)
        elif isinstance(allocator, _TorchAllocator):
            self._allocator = allocator
        elif allocator != "cuda":
            raise ValueError(allocator)
        if self._allocator is not None:
            opt.alloc = self._allocator.alloc
            opt.free = self._allocator.free
        opt.member_slots = int(member_slots)
        opt.warp_max_degree = int(warp_max_degree)
        opt.use_graphs = 0 if use_graphs else -1
        opt.profile = 1 if profile else 0
        opt.exhaustive_fp64 = 1 if exhaustive_fp64 else 0
        # True: launches per queue; False: persistent loop; None: by queue size
        opt.per_queue_launches = 0 if per_queue_launches is None else (1 if per_queue_launches else 2)
        opt.barrier_timeout_ms = int(barrier_timeout_ms)
        opt.inject_barrier_stall = 1 if inject_barrier_stall else 0
        opt.barrier_mode = int(barrier_mode)
        opt.warps_per_node = int(warps_per_node)
        opt.hub_degree = int(hub_degree)
        if gain_rule not in GAIN_RULES:
            raise ValueError(f"unknown gain_rule {gain_rule!r}")
        opt.gain_rule = GAIN_RULES[gain_rule]
        opt.debug_checks = 1 if debug_checks else 0
        if isinstance(src, torch.Tensor):
            if src.dtype != torch.int32 or dst.dtype != torch.int32 or not src.is_cuda:
                raise TypeError("device edge lists must be int32 CUDA tensors")
            src = src.contiguous()
            dst = dst.contiguous()
            opt.edges_on_device = 1
            E = src.numel()
            ps, pd = C.c_void_p(src.data_ptr()), C.c_void_p(dst.data_ptr())
            keep = (src, dst)
        else:
            src = np.ascontiguousarray(src, dtype=np.int32)
            dst = np.ascontiguousarray(dst, dtype=np.int32)
            if src.shape != dst.shape:
                raise ValueError("src and dst differ in length")
            opt.edges_on_device = 0
            E = src.shape[0]
            ps, pd = C.c_void_p(src.ctypes.data), C.c_void_p(dst.ctypes.data)
            keep = (src, dst)
        self._opt = opt
        if edge_offsets is None:
            _check(self._L, self._L.lf_graph_create(ps, pd, E, C.byref(opt), C.byref(self._h)))
        else:   # a batch of graphs (host edge lists only)
            if opt.edges_on_device:
                raise TypeError("a batch takes host edge lists")
            eo = np.ascontiguousarray(edge_offsets, dtype=np.int64)
            _check(self._L, self._L.lf_batch_create(ps, pd, _ptr(eo, C.c_int64), eo.shape[0] - 1, C.byref(opt),
                                                    C.byref(self._h)))
        del keep
        n, m = C.c_int64(), C.c_int64()
        _check(self._L, self._L.lf_get_sizes(self._h, C.byref(n), C.byref(m)))
        self.n, self.m = n.value, m.value

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.lf_graph_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the method -----------------------------------------------------------
    def autotune(self, queue_size: int, trial_iters: int = 1) -> dict:
        """Choose the launch shape of the later runs by timing short runs
        (lf_autotune); returns the choice and the trial times."""
        r = TuneResultC()
        _check(self._L, self._L.lf_autotune(self._h, int(queue_size), int(trial_iters), C.byref(r)))
        return dict(warps_per_node=r.warps_per_node, warp_max_degree=r.warp_max_degree,
                    hub_degree=r.hub_degree, trials=r.trials,
                    best_ms=r.best_ms, default_ms=r.default_ms)

    def set_partition(self, communities):
        """Insert a division that replaces the initial clustering of the next
        runs: a list of arrays of original node ids (may overlap), or an
        (offsets, members) pair as `communities()` returns; None removes it."""
        if communities is None:
            _check(self._L, self._L.lf_set_partition(self._h, None, None, -1))
            return
        if isinstance(communities, tuple) and len(communities) == 2 and np.ndim(communities[0]) == 1 \
                and np.asarray(communities[0]).dtype.kind == "i" and not isinstance(communities[0], list):
            off = np.ascontiguousarray(communities[0], dtype=np.int64)
            mem = np.ascontiguousarray(communities[1], dtype=np.int32)
        else:
            sizes = np.array([len(c) for c in communities], dtype=np.int64)
            off = np.zeros(sizes.shape[0] + 1, dtype=np.int64)
            np.cumsum(sizes, out=off[1:])
            mem = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int32) for c in communities])
                                       if len(communities) else np.zeros(0, np.int32))
        if mem.shape[0] == 0:
            mem = np.zeros(1, np.int32)
        _check(self._L, self._L.lf_set_partition(self._h, _ptr(off, C.c_int64), _ptr(mem, C.c_int32),
                                                 off.shape[0] - 1))

    def run(self, queue_size: int, wcc_threshold: float = 0.01, max_iters: int = 50,
            max_batches: int | None = None, on_iteration=None) -> RunStats:
        """on_iteration(iteration, wcc) is called after every iteration; it may
        call communities() (the intermediate result) and returns True to stop."""
        cb = None
        if on_iteration is None:
            on_iteration = getattr(self, "_on_iteration", None)   # set by lf_set_iteration_callback
        if on_iteration is not None:
            def _tramp(_g, it, wcc, _ctx):
                try:
                    return 1 if on_iteration(int(it), float(wcc)) else 0
                except Exception:  # noqa: BLE001 - stop the run; the error is re-raised below
                    import sys
                    self._cb_error = sys.exc_info()[1]
                    return 1
            cb = _ITER_FN(_tramp)
            self._cb_error = None
            _check(self._L, self._L.lf_set_iteration_callback(self._h, cb, None))
        try:
            return self._run(queue_size, wcc_threshold, max_iters, max_batches)
        finally:
            if cb is not None:
                self._L.lf_set_iteration_callback(self._h, _ITER_FN(), None)
                if self._cb_error is not None:
                    err, self._cb_error = self._cb_error, None
                    raise err

    def _run(self, queue_size, wcc_threshold, max_iters, max_batches) -> RunStats:
        cap = max(1, max_iters)
        T = np.zeros(cap, np.float64)
        J = np.zeros(cap, np.int64)
        Lv = np.zeros(cap, np.int64)
        st = RunStatsC()
        st.history_cap = cap
        st.wcc_history = _ptr(T, C.c_double)
        st.joins_history = _ptr(J, C.c_int64)
        st.leaves_history = _ptr(Lv, C.c_int64)
        if max_batches is None:
            s = self._L.lf_run(self._h, int(queue_size), float(wcc_threshold), int(max_iters), C.byref(st))
        else:
            s = self._L.lf_run_partial(self._h, int(queue_size), float(wcc_threshold), int(max_iters),
                                       int(max_batches), C.byref(st))
        _check(self._L, s)
        k = st.iterations
        return RunStats(k, bool(st.converged), st.num_batches, st.wcc_initial, T[:k].copy(), J[:k].copy(),
                        Lv[:k].copy(), st.num_communities, st.num_memberships, st.ms_total, st.ms_init,
                        st.ms_iterations, st.num_launches, st.prof_move_launches, st.prof_move_ms,
                        st.prof_move_bytes, tuple(st.prof_queue_us), st.prof_candidates, st.prof_exact)

    def communities(self):
        """(offsets int64[k+1], members int32[...]) in original node ids."""
        nc, nm = C.c_int64(), C.c_int64()
        _check(self._L, self._L.lf_get_communities(self._h, None, 0, None, 0, C.byref(nc), C.byref(nm)))
        off = np.zeros(nc.value + 1, np.int64)
        mem = np.zeros(max(1, nm.value), np.int32)
        _check(self._L, self._L.lf_get_communities(self._h, _ptr(off, C.c_int64), off.shape[0],
                                                   _ptr(mem, C.c_int32), mem.shape[0],
                                                   C.byref(nc), C.byref(nm)))
        return off, mem[:nm.value]

    def community_list(self):
        off, mem = self.communities()
        return [mem[off[i]:off[i + 1]] for i in range(off.shape[0] - 1)]

    # -- inspection -------------------------------------------------------------
    def node_stats(self):
        t = np.zeros(max(1, self.n), np.int64)
        vt = np.zeros(max(1, self.n), np.int32)
        cc = C.c_double()
        _check(self._L, self._L.lf_get_node_stats(self._h, _ptr(t, C.c_int64), _ptr(vt, C.c_int32), C.byref(cc)))
        return t[:self.n], vt[:self.n], cc.value

    def csr(self):
        off = np.zeros(self.n + 1, np.int64)
        adj = np.zeros(max(1, 2 * self.m), np.int32)
        labels = np.zeros(max(1, self.n), np.int32)
        _check(self._L, self._L.lf_get_csr(self._h, _ptr(off, C.c_int64), _ptr(adj, C.c_int32),
                                           _ptr(labels, C.c_int32)))
        return off, adj[:2 * self.m], labels[:self.n]

    def oriented(self):
        off = np.zeros(self.n + 1, np.int64)
        adj = np.zeros(max(1, self.m), np.int32)
        _check(self._L, self._L.lf_get_oriented(self._h, _ptr(off, C.c_int64), _ptr(adj, C.c_int32)))
        return off, adj[:self.m]

    def order(self):
        o = np.zeros(max(1, self.n), np.int32)
        _check(self._L, self._L.lf_get_order(self._h, _ptr(o, C.c_int32)))
        return o[:self.n]

    def state(self):
        nm, nc = C.c_int64(), C.c_int64()
        _check(self._L, self._L.lf_get_state(self._h, None, None, None, None, None, C.byref(nm), C.byref(nc)))
        mem_off = np.zeros(self.n + 1, np.int64)
        mem_ids = np.zeros(max(1, nm.value), np.int32)
        cn = np.zeros(max(1, nc.value), np.int64)
        cm = np.zeros(max(1, nc.value), np.int64)
        cv = np.zeros(max(1, nc.value), np.int64)
        _check(self._L, self._L.lf_get_state(self._h, _ptr(mem_off, C.c_int64), _ptr(mem_ids, C.c_int32),
                                             _ptr(cn, C.c_int64), _ptr(cm, C.c_int64), _ptr(cv, C.c_int64),
                                             C.byref(nm), C.byref(nc)))
        k = nc.value
        return dict(mem_off=mem_off, mem_ids=mem_ids[:nm.value], n=cn[:k], m=cm[:k], vol=cv[:k])

    def create_stats(self) -> dict:
        s = CreateStatsC()
        _check(self._L, self._L.lf_get_create_stats(self._h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in CreateStatsC._fields_}


def run_lazyfox(src, dst, queue_size: int, wcc_threshold: float = 0.01, max_iters: int = 50, **kw):
    """One call end to end: build, run, return (communities, stats)."""
    with Graph(src, dst, **kw) as g:
        st = g.run(queue_size, wcc_threshold, max_iters)
        return g.community_list(), st


def infinity_threshold() -> float:
    return -math.inf


class Batch(Graph):
    """Many independent graphs run together (``lf_batch_create``): every launch
    of a run covers all of them, and each graph gets exactly the result it
    would get alone.  ``graphs``: a list of (src, dst) int32 host arrays or of
    objects with ``src``/``dst``.  Other keywords as for :class:`Graph`."""

    def __init__(self, graphs, **kw):
        pairs = [(g.src, g.dst) if hasattr(g, "src") else g for g in graphs]
        sizes = np.array([len(p[0]) for p in pairs], dtype=np.int64)
        off = np.zeros(len(pairs) + 1, dtype=np.int64)
        np.cumsum(sizes, out=off[1:])
        src = np.concatenate([np.asarray(p[0], dtype=np.int32) for p in pairs]) if pairs else np.zeros(0, np.int32)
        dst = np.concatenate([np.asarray(p[1], dtype=np.int32) for p in pairs]) if pairs else np.zeros(0, np.int32)
        self.num_graphs = len(pairs)
        super().__init__(src, dst, edge_offsets=off, **kw)

    def info(self):
        """Per graph: node offsets in the union, iterations, converged,
        WCC-hat after the initial clustering and at the end, cc."""
        G = self.num_graphs
        ng = C.c_int64()
        noff = np.zeros(G + 1, np.int64)
        it = np.zeros(G, np.int32)
        conv = np.zeros(G, np.int32)
        t0 = np.zeros(G, np.float64)
        tf = np.zeros(G, np.float64)
        cc = np.zeros(G, np.float64)
        _check(self._L, self._L.lf_batch_get_info(self._h, C.byref(ng), _ptr(noff, C.c_int64), _ptr(it, C.c_int32),
                                                  _ptr(conv, C.c_int32), _ptr(t0, C.c_double),
                                                  _ptr(tf, C.c_double), _ptr(cc, C.c_double)))
        return dict(node_offsets=noff, iterations=it, converged=conv.astype(bool), wcc_initial=t0,
                    wcc_final=tf, cc=cc)

    def history(self, graph: int):
        cnt = C.c_int32()
        _check(self._L, self._L.lf_batch_get_history(self._h, int(graph), None, 0, C.byref(cnt)))
        h = np.zeros(max(1, cnt.value), np.float64)
        _check(self._L, self._L.lf_batch_get_history(self._h, int(graph), _ptr(h, C.c_double), h.shape[0],
                                                     C.byref(cnt)))
        return h[:cnt.value]

    def graph_communities(self):
        """For every graph, its communities as arrays of its own node ids."""
        nc, nm = C.c_int64(), C.c_int64()
        _check(self._L, self._L.lf_batch_get_communities(self._h, None, None, 0, None, 0, C.byref(nc), C.byref(nm)))
        goff = np.zeros(self.num_graphs + 1, np.int64)
        off = np.zeros(nc.value + 1, np.int64)
        mem = np.zeros(max(1, nm.value), np.int32)
        _check(self._L, self._L.lf_batch_get_communities(self._h, _ptr(goff, C.c_int64), _ptr(off, C.c_int64),
                                                         off.shape[0], _ptr(mem, C.c_int32), mem.shape[0],
                                                         C.byref(nc), C.byref(nm)))
        return [[mem[off[c]:off[c + 1]] for c in range(goff[i], goff[i + 1])] for i in range(self.num_graphs)]


class Server:
    """Serving with continuous batching (``lf_server_*``): submit graphs at any
    time; admitted jobs stay resident and run side by side on the device."""

    def __init__(self, hbm_budget_bytes: int = 0, max_active: int = 4):
        self._L = load_library()
        self._h = C.c_void_p()
        opt = ServerOptionsC(int(hbm_budget_bytes), int(max_active), 0)
        _check(self._L, self._L.lf_server_create(C.byref(opt), C.byref(self._h)))

    def submit(self, src, dst, queue_size: int, wcc_threshold: float = 0.01, max_iters: int = 50) -> int:
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        jid = C.c_int64()
        _check(self._L, self._L.lf_server_submit(self._h, C.c_void_p(src.ctypes.data), C.c_void_p(dst.ctypes.data),
                                                 src.shape[0], int(queue_size), float(wcc_threshold),
                                                 int(max_iters), C.byref(jid)))
        return jid.value

    def wait(self, job: int, timeout_s: float = -1.0) -> dict:
        r = JobResultC()
        _check(self._L, self._L.lf_server_wait(self._h, int(job), float(timeout_s), C.byref(r)))
        return {k: getattr(r, k) for k, _ in JobResultC._fields_ if k != "pad"}

    def community_list(self, job: int):
        nc, nm = C.c_int64(), C.c_int64()
        _check(self._L, self._L.lf_server_get_communities(self._h, int(job), None, 0, None, 0, C.byref(nc),
                                                          C.byref(nm)))
        off = np.zeros(nc.value + 1, np.int64)
        mem = np.zeros(max(1, nm.value), np.int32)
        _check(self._L, self._L.lf_server_get_communities(self._h, int(job), _ptr(off, C.c_int64), off.shape[0],
                                                          _ptr(mem, C.c_int32), mem.shape[0], C.byref(nc),
                                                          C.byref(nm)))
        return [mem[off[i]:off[i + 1]] for i in range(nc.value)]

    def release(self, job: int):
        _check(self._L, self._L.lf_server_release(self._h, int(job)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.lf_server_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def _cover_csr(cover):
    if isinstance(cover, tuple) and len(cover) == 2 and not isinstance(cover[0], list):
        return np.ascontiguousarray(cover[0], dtype=np.int64), np.ascontiguousarray(cover[1], dtype=np.int32)
    sizes = np.array([len(c) for c in cover], dtype=np.int64)
    off = np.zeros(len(cover) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    mem = (np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int32) for c in cover]))
           if len(cover) and off[-1] > 0 else np.zeros(0, np.int32))
    return off, mem


def cover_f1(detected, reference, stream=None):
    """F1-score of a detected cover against a reference cover (``lf_cover_f1``,
    on the GPU): covers as lists of id arrays or (offsets, members).  Returns
    (f1, best reference index per detected community)."""
    L = load_library()
    oa, ma = _cover_csr(detected)
    ob, mb = _cover_csr(reference)
    ka, kb = oa.shape[0] - 1, ob.shape[0] - 1
    ma1 = ma if ma.shape[0] else np.zeros(1, np.int32)
    mb1 = mb if mb.shape[0] else np.zeros(1, np.int32)
    f = C.c_double()
    best = np.zeros(max(1, ka), np.int32)
    st = C.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(L, L.lf_cover_f1(_ptr(oa, C.c_int64), _ptr(ma1, C.c_int32), ka, _ptr(ob, C.c_int64), _ptr(mb1, C.c_int32),
                            kb, C.byref(f), _ptr(best, C.c_int32), st))
    return f.value, best[:ka]


def quality_report(el, queue_sizes=(2, 4, 8, 16, 32, 64, 128, 256), threshold: float = 0.01, max_iters: int = 50):
    """F1 of LazyFox at each queue size against Fox (queue size 1) and, when
    the graph has one, against its planted cover; Fox against the planted
    cover too (the comparison of the paper's quality table)."""
    def detect(q):
        with Graph(el.src, el.dst) as g:
            g.run(q, threshold, max_iters)
            return g.communities()
    fox = detect(1)
    planted = None
    if getattr(el, "planted", None) is not None:
        planted = [np.unique(np.asarray(c, dtype=np.int32)) for c in el.planted]
        planted = [c for c in planted if c.shape[0]]
    rows = [dict(queue_size=1, f1_vs_fox=1.0 if fox[0].shape[0] > 1 else 0.0,
                 f1_vs_planted=cover_f1(fox, planted)[0] if planted else None)]
    for q in queue_sizes:
        lazy = detect(q)
        rows.append(dict(queue_size=q, f1_vs_fox=cover_f1(lazy, fox)[0],
                         f1_vs_planted=cover_f1(lazy, planted)[0] if planted else None))
    return rows


# -- the entry points of include/lazyfox.h under their own names ---------------
# One thin function per entry point: a handle is a Graph, Batch or Server
# object; host buffers are numpy arrays, device buffers int32/int64 CUDA
# tensors.  Each marshals its arguments and reaches the entry point of the
# same name (through the methods above, which do the marshalling).

def lf_graph_create(src, dst, **options) -> Graph:
    """Build a graph and run the preprocessing; options as for :class:`Graph`."""
    return Graph(src, dst, **options)


def lf_run(g: Graph, queue_size: int, wcc_threshold: float = 0.01, max_iters: int = 50) -> RunStats:
    return g.run(queue_size, wcc_threshold, max_iters)


def lf_run_partial(g: Graph, queue_size: int, wcc_threshold: float, max_iters: int, max_batches: int) -> RunStats:
    return g.run(queue_size, wcc_threshold, max_iters, max_batches=max_batches)


def lf_get_communities(g: Graph):
    """(offsets int64[k+1], members int32[...]) in original node ids."""
    return g.communities()


def lf_get_node_stats(g: Graph):
    """(t int64[n], vt int32[n], cc)."""
    return g.node_stats()


def lf_get_sizes(g: Graph):
    """(nodes n, undirected simple edges m)."""
    n, m = C.c_int64(), C.c_int64()
    _check(g._L, g._L.lf_get_sizes(g._h, C.byref(n), C.byref(m)))
    return n.value, m.value


def lf_get_create_stats(g: Graph) -> dict:
    return g.create_stats()


def lf_get_csr(g: Graph):
    """(offsets int64[n+1], neighbours int32[2m], labels int32[n])."""
    return g.csr()


def lf_get_oriented(g: Graph):
    return g.oriented()


def lf_get_order(g: Graph):
    return g.order()


def lf_get_state(g: Graph) -> dict:
    return g.state()


def lf_graph_destroy(g: Graph) -> None:
    g.close()


def lf_last_error() -> str:
    """The calling thread's message of its last failed call."""
    return load_library().lf_last_error().decode(errors="replace")


def lf_triangles_noalloc(ooff, oadj, t, vt, stream=None) -> None:
    """t(x,V) and vt(x,V) of an oriented CSR (device tensors: ooff int64[n+1],
    oadj int32[m]) into device tensors t int64[n] and vt int32[n], without any
    device allocation (``stream``: a torch.cuda.Stream; default torch's
    current stream)."""
    import torch
    for a, dt in ((ooff, torch.int64), (oadj, torch.int32), (t, torch.int64), (vt, torch.int32)):
        if not isinstance(a, torch.Tensor) or a.dtype != dt or not a.is_cuda or not a.is_contiguous():
            raise TypeError("lf_triangles_noalloc takes contiguous CUDA tensors: ooff int64, oadj int32, "
                            "t int64, vt int32")
    n = ooff.numel() - 1
    if n < 0 or t.numel() < n or vt.numel() < n:
        raise ValueError("ooff needs n+1 entries and t, vt n each")
    L = load_library()
    # default: torch's current stream, so that work queued there before the
    # call (e.g. the writes of the inputs) is ordered before it
    st = C.c_void_p((stream if stream is not None else torch.cuda.current_stream(ooff.device)).cuda_stream)
    _check(L, L.lf_triangles_noalloc(C.c_void_p(ooff.data_ptr()), C.c_void_p(oadj.data_ptr()), n, oadj.numel(),
                                     C.c_void_p(t.data_ptr()), C.c_void_p(vt.data_ptr()), st))


def lf_set_partition(g: Graph, communities) -> None:
    g.set_partition(communities)


def lf_set_iteration_callback(g: Graph, fn) -> None:
    """fn(iteration, wcc) after every iteration of g's later runs (True stops
    the run); None removes it."""
    g._on_iteration = fn


def lf_batch_create(graphs, **options) -> Batch:
    return Batch(graphs, **options)


def lf_batch_get_info(b: Batch) -> dict:
    return b.info()


def lf_batch_get_history(b: Batch, graph: int):
    return b.history(graph)


def lf_batch_get_communities(b: Batch):
    """For every graph, its communities as arrays of its own node ids."""
    return b.graph_communities()


def lf_autotune(g: Graph, queue_size: int, trial_iters: int = 1) -> dict:
    return g.autotune(queue_size, trial_iters)


def lf_server_create(hbm_budget_bytes: int = 0, max_active: int = 4) -> Server:
    return Server(hbm_budget_bytes, max_active)


def lf_server_submit(s: Server, src, dst, queue_size: int, wcc_threshold: float = 0.01, max_iters: int = 50) -> int:
    return s.submit(src, dst, queue_size, wcc_threshold, max_iters)


def lf_server_wait(s: Server, job: int, timeout_s: float = -1.0) -> dict:
    return s.wait(job, timeout_s)


def lf_server_get_communities(s: Server, job: int):
    return s.community_list(job)


def lf_server_release(s: Server, job: int) -> None:
    s.release(job)


def lf_server_destroy(s: Server) -> None:
    s.close()


def lf_cover_f1(detected, reference, stream=None):
    """(F1, best reference index per detected community)."""
    return cover_f1(detected, reference, stream)
