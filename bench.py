#!/usr/bin/env python3
"""Benchmark of the LazyFox hot path on one GB300 (or N replicas).

One step = the whole hot path on one synthetic graph: lf_graph_create
(self-loop/duplicate removal, relabel, CSR, orientation, triangles, vt, node
order, cc) followed by lf_run (initial clustering, then LazyFox iterations of
move evaluation + bulk apply per queue, pruning and the exact WCC-hat total,
until the relative change falls below the threshold).

value      = edges/s per iteration: m x iterations / step time, summed over the
             timed steps (device-resident input, CUDA events on the library's
             stream, L2 flushed by a 256 MiB write before every step).
e2e        = the same metric through the public API from pinned host buffers:
             host->device copy of the edge list, the run, and the device->host
             read of the communities inside the timed region.
roofline   = the move-evaluation kernel (the dominant kernel): algorithmic bytes
             per launch / mean launch time (CUDA events around every launch in
             the timed steps) against the measured HBM copy bandwidth.
cpu_baseline = the sequential CPU oracle on the same workload (rank 0, N=1).

--impl reference times the CPU oracle as the reference arm.
Under torchrun every rank runs its own replica (no collective on the data
path); value = edges x iterations of all ranks / max over ranks of the time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "edges/s per Fox iteration + triangle-count GB/s; batched graphs/s & p99 vs plain"
UNIT = "edges/s per iteration"
FALLBACK_HBM_GBS = 6800.0

# cpu_sample: the bounded sample of the workload the oracle is timed on (the
# cpu_baseline leg and the reference arm), when a whole run is too long.
WORKLOADS = {
    # 3.07M nodes, ~115M edges, Chung-Lu gamma 2.2, max degree ~33k, planted
    # communities of 10-5,000 nodes; queue size 65536, 20 iterations
    "large": dict(name="large_like_3.07M_nodes_115M_edges", gen=("large_like", {}), q=65536,
                  threshold=-math.inf, max_iters=20,
                  cpu_sample=dict(gen=("large_like", {"scale": 0.02}), max_iters=1,
                                  what="the same generator at 2% scale (61,400 nodes, 2.07M edges): preprocessing "
                                       "and the first iteration at queue size 65536 (one queue holds every node)"),
                  secondary=[dict(workload="large", q=65536, rule="meanfield"),
                             dict(workload="dblp", q=1024, rule="literal"),
                             dict(workload="dblp", q=64, rule="literal"),
                             dict(workload="dblp", q=1024, rule="meanfield")]),
    # the same generator at a quarter of the nodes (767,500 nodes, ~29M
    # edges), queue size 16384, 20 iterations: the size detailed ncu captures
    # of the move-evaluation kernels are taken on
    "large_quarter": dict(name="large_like_767k_nodes_quarter_scale", gen=("large_like", {"scale": 0.25}), q=16384,
                          threshold=-math.inf, max_iters=20,
                          cpu_sample=dict(gen=("large_like", {"scale": 0.02}), max_iters=1,
                                          what="the same generator at 2% scale (61,400 nodes, 2.07M edges): "
                                               "preprocessing and the first iteration at queue size 16384"),
                          secondary=[]),
    # 335k nodes, ~0.93M edges, Chung-Lu gamma 2.5, max degree ~550, planted
    # overlapping communities (sizes 6-2,000, 1-4 per node), seed 1
    "dblp": dict(name="dblp_like_335k_nodes_0.93M_edges", gen=("dblp_like", {}), q=1024, threshold=0.01,
                 max_iters=50, cpu_sample=None,
                 secondary=[dict(workload="dblp", q=64, rule="literal"),
                            dict(workload="dblp", q=1024, rule="meanfield")]),
    # 1,000 nodes, 20 planted communities, Fox (queue size 1)
    "eu": dict(name="eu_core_like_1k_nodes_planted_er", gen=("eu_core_like", {}), q=1, threshold=0.01,
               max_iters=50, cpu_sample=None, secondary=[]),
    # 4,096 planted graphs, nodes log-uniform 200-20k, average degree 8-40,
    # one batch per step against one graph per call
    "batched": dict(name="batched_planted_graphs_200-20k_nodes_deg_8-40", gen=None, q=256,
                    threshold=0.01, max_iters=50),
    # Poisson stream of planted graphs, nodes log-uniform 1k-2M, degree 10-80
    "serving": dict(name="serving_poisson_planted_graphs_1k-2M_nodes_deg_10-80", gen=None, q=1024,
                    threshold=0.01, max_iters=50),
}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lazyfox", "reference"], default="lazyfox")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--gain-rule", choices=["literal", "meanfield"], default="literal",
                    help="decision rule of a move: the paper's gain (change of WCC-hat(P)) or the mean-field departure")
    ap.add_argument("--queue-size", type=int, default=None)
    ap.add_argument("--no-secondary", action="store_true", help="skip the secondary lines (other rule, other workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-graphs", type=int, default=4096, help="graphs per batch (batched workload)")
    ap.add_argument("--jobs", type=int, default=48, help="jobs of the serving stream")
    ap.add_argument("--rate", type=float, default=200.0, help="mean arrivals per second (serving)")
    ap.add_argument("--max-nodes", type=int, default=200_000,
                    help="largest job (serving; the full 1k-2M range generates ~1e9 edges on the host)")
    ap.add_argument("--max-active", type=int, default=4, help="jobs resident at once (serving)")
    ap.add_argument("--plain-sample", type=int, default=256,
                    help="graphs run one per call for the plain comparison (batched workload)")
    return ap.parse_args()


def make_workload(spec):
    from paper_2210_03211_gb300 import workloads as W
    fn, kw = spec["gen"]
    return getattr(W, fn)(**kw)


def cpu_sample_graph(spec):
    """The graph the oracle is timed on, its iteration limit and what it is."""
    smp = spec.get("cpu_sample")
    if smp is None:
        return make_workload(spec), spec["max_iters"], "one full run (preprocessing and every iteration) of the workload"
    return make_workload(smp), smp["max_iters"], smp["what"]


def measured_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001 - absent or unreadable: the recipe's fallback
        return FALLBACK_HBM_GBS, "fallback"


def ncu_traffic(kernel: str, workload: str, queue_size: int):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source has not changed since it was captured and the summary is for this
    workload and queue size (a launch's traffic depends on both)."""
    import hashlib
    summ = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    if not os.path.exists(summ):
        return None
    vals = {}
    for line in open(summ):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2210_03211_gb300", "csrc", vals.get("source", "lf_run.cu"))
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if vals.get("source_sha256_16") != sha:
        return None
    if vals.get("bench_workload") != workload or vals.get("bench_queue_size") != str(queue_size):
        return None
    try:
        return dict(bytes_per_launch=float(vals["dram_bytes_per_launch_scaled"]),
                    workload=vals.get("captured_on", ""))
    except (KeyError, ValueError):
        return None


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(use_gpu_backend: bool):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if use_gpu_backend else "gloo")
    return rank, world, local


def reduce_max(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def time_oracle(el, q, threshold, max_iters, rule="literal"):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    og = oracle.OracleGraph(el.src, el.dst)
    r = og.run(q, threshold, max_iters, rule=rule)
    dt = time.perf_counter() - t0
    return og.m * r["iterations"], dt, r["iterations"]


def _oracle_worker_ready(_):
    import oracle
    oracle.lib()
    time.sleep(0.2)   # holds this worker so that every worker takes one
    return os.getpid()


def _oracle_graph_seconds(job):
    src, dst, q, threshold, max_iters, rule = job
    import oracle
    t0 = time.perf_counter()
    og = oracle.OracleGraph(src, dst)
    og.run(q, threshold, max_iters, rule=rule)
    return time.perf_counter() - t0


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_info() -> dict:
    """The host a CPU baseline ran on: the logical CPUs this process may use,
    the architecture and the CPU model as lscpu names it (None if unknown)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:  # noqa: BLE001 - no lscpu: the model stays unknown
        pass
    return {"nproc": host_cores(), "machine": platform.machine(), "cpu_model": model}


def oracle_graphs_per_s(graphs, q, threshold, max_iters, cores, rule="literal"):
    """The oracle on independent graphs, one process per host core: a 'spawn'
    pool (safe after GPU calls), every worker started and the oracle loaded
    before the clock starts, the largest graphs handed out first.  Returns
    graphs / wall time of the whole sample and the CPU seconds it took."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    jobs = sorted(((g.src, g.dst, q, threshold, max_iters, rule) for g in graphs), key=lambda j: -j[0].shape[0])
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_worker_ready, range(cores), chunksize=1)
        t0 = time.perf_counter()
        secs = list(pool.imap_unordered(_oracle_graph_seconds, jobs, chunksize=1))
        wall = time.perf_counter() - t0
    return len(jobs) / wall, sum(secs)


def oracle_batch_sample(graphs, cores):
    """The CPU baseline's sample of a batch: its first 2 x cores graphs of at
    most 5,000 nodes (the paper's gain costs the oracle a pass over each
    candidate community, so larger planted graphs take minutes each)."""
    out = []
    for g in graphs:
        if np.unique(np.concatenate([g.src, g.dst])).shape[0] <= 5000:
            out.append(g)
            if len(out) == max(8, 2 * cores):
                break
    return out


def run_reference(args, spec, q):
    rank, world, _ = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), 0
    if rank != 0:
        return 0
    if spec["gen"] is None:   # batched / serving: the oracle on a sample of the graphs, one process per core
        from paper_2210_03211_gb300 import workloads as W
        cores = host_cores()
        graphs = (oracle_batch_sample(W.batched_planted(args.batch_graphs, seed=5), cores)
                  if args.workload == "batched" else W.serving_jobs(max(8, cores), seed=7, n_hi=5000)[0])
        value, cpu_s = oracle_graphs_per_s(graphs, q, spec["threshold"], spec["max_iters"], cores, args.gain_rule)
        what = ("batch with at most 5,000 nodes" if args.workload == "batched"
                else "job stream (nodes capped at 5k)")
        line = {"metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": args.gpus, "steps": 1,
                "warmup": 0, "ms_per_step": 1e3 * len(graphs) / value, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64", "data": "synthetic",
                "impl": "reference",
                "config": {"workload": spec["name"], "graphs": len(graphs), "queue_size": q},
                "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": cores, "kind": "oracle",
                                 "sample": f"the first {len(graphs)} graphs of the {what}, one oracle process "
                                           f"per host core ({cpu_s:.1f} CPU seconds)", "host": host_info()},
                "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    el, max_iters, what = cpu_sample_graph(spec)
    for _ in range(min(args.warmup, 1)):   # the oracle has no caches to warm; one untimed run loads it
        time_oracle(el, q, spec["threshold"], max_iters, args.gain_rule)
    units, secs, iters = 0.0, 0.0, []
    for _ in range(args.steps):
        u, dt, it = time_oracle(el, q, spec["threshold"], max_iters, args.gain_rule)
        units += u
        secs += dt
        iters.append(it)
    value = units / secs
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": spec["name"], "queue_size": q, "threshold": spec["threshold"],
                   "max_iters": spec["max_iters"], "gain_rule": args.gain_rule, "iterations": iters},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: {what}", "host": host_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, spec, q):
    """Graphs per second of one batch (lf_batch_create + lf_run + the
    communities of every graph) against the same graphs one per call
    (lf_graph_create + lf_run + lf_get_communities); latency percentiles of
    the plain calls and of the batch (every graph of a batch finishes with it)."""
    import numpy as np
    import torch

    from paper_2210_03211_gb300 import build as lf_build
    from paper_2210_03211_gb300 import lazyfox
    from paper_2210_03211_gb300 import workloads as W

    rank, world, local = dist_setup(torch.cuda.is_available())
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU: the library has no CPU path")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        lf_build.build()
    barrier(world)
    lazyfox.load_library()
    graphs = W.batched_planted(args.batch_graphs, seed=5 + rank)
    G = len(graphs)
    edges = sum(int(g.src.shape[0]) for g in graphs)
    stream = torch.cuda.Stream(dev)
    # the launch shape, chosen once by the library's autotuner on this batch
    rule = args.gain_rule
    with lazyfox.Batch(graphs, stream=stream, gain_rule=rule) as b:
        tune = b.autotune(q, 1)
    shape = dict(warps_per_node=tune["warps_per_node"], warp_max_degree=tune["warp_max_degree"],
                 hub_degree=tune["hub_degree"])

    def batch_step():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with lazyfox.Batch(graphs, stream=stream, gain_rule=rule, **shape) as b:
            b.run(q, spec["threshold"], spec["max_iters"])
            comms = b.graph_communities()
            it = b.info()["iterations"]
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1), comms, it

    for _ in range(args.warmup):
        batch_step()
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks_s = ClockSampler("GPU-" + str(torch.cuda.get_device_properties(dev).uuid))
    clocks_s.start()
    res = [batch_step() for _ in range(args.steps)]
    clocks = clocks_s.stop()
    torch.cuda.synchronize(dev)
    barrier(world)
    local_ms = sum(r[0] for r in res)
    total_ms = reduce_max(local_ms, world, dev)
    value = reduce_sum(G * len(res), world, dev) / (total_ms / 1e3)
    # plain: one graph per call, on a sample of the same graphs
    sample = graphs[:max(1, min(args.plain_sample, G))]
    lat = []
    for el in sample[:2]:   # warm-up
        with lazyfox.Graph(el.src, el.dst, stream=stream, gain_rule=rule) as g:
            g.run(q, spec["threshold"], spec["max_iters"])
            g.communities()
    for el in sample:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with lazyfox.Graph(el.src, el.dst, stream=stream, gain_rule=rule) as g:
            g.run(q, spec["threshold"], spec["max_iters"])
            g.communities()
            e1.record(stream)
        stream.synchronize()
        lat.append(e0.elapsed_time(e1))
    lat = np.array(lat)
    plain_gps = len(lat) / (lat.sum() / 1e3)
    # the sampled graphs' results, alone and in the batch, must agree
    same = True
    for i, el in enumerate(sample[:32]):
        with lazyfox.Graph(el.src, el.dst, stream=stream, gain_rule=rule) as g:
            g.run(q, spec["threshold"], spec["max_iters"])
            same &= [c.tolist() for c in g.community_list()] == [c.tolist() for c in res[-1][1][i]]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        cpu_sample = oracle_batch_sample(graphs, cores)
        cpu_gps, cpu_s = oracle_graphs_per_s(cpu_sample, q, spec["threshold"], spec["max_iters"], cores, rule)
        cpu = {"value": cpu_gps, "unit": "graphs/s", "cores": cores, "kind": "oracle",
               "sample": f"the first {len(cpu_sample)} graphs of the batch with at most 5,000 nodes, one oracle "
                         f"process per host core ({cpu_s:.1f} CPU seconds; gain rule {rule})", "host": host_info()}
    if rank == 0:
        batch_ms = np.array([r[0] for r in res])
        line = {
            "metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64", "data": "synthetic",
            "config": {"workload": spec["name"], "graphs": G, "edges": edges, "queue_size": q, "gain_rule": rule,
                       "threshold": spec["threshold"], "max_iters": spec["max_iters"],
                       "iterations_max": int(max(res[-1][2])), "parallelism": f"replicas x{world}",
                       "timed": "lf_batch_create (host edge lists, copied in) + lf_run + communities of every graph",
                       "l2": "inputs (~GB) larger than L2"},
            "autotune": tune,
            "plain": {"graphs_per_s": plain_gps, "sample": len(lat), "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)),
                      "timed": "lf_graph_create + lf_run + lf_get_communities, one graph per call"},
            "batched": {"graphs_per_s": value, "p50_ms": float(np.percentile(batch_ms, 50)),
                        "p99_ms": float(np.percentile(batch_ms, 99)), "speedup_vs_plain": value / plain_gps},
            "results_equal_alone_and_batched": bool(same),
            "cpu_baseline": cpu,
            "clocks": clocks,
            "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": int(8 * edges),
                    "d2h_bytes_per_step": None, "note": "the batched step already starts from host edge lists"},
        }
        print(json.dumps(line), flush=True)
    return 0


def fifo_finish(arrivals, service):
    """Finish times of jobs served one at a time in arrival order (first
    come, first served): each starts at its arrival or when the previous one
    finishes, whichever is later."""
    import numpy as np
    fin = np.zeros(len(arrivals))
    for i in range(len(arrivals)):
        start = max(arrivals[i], fin[i - 1] if i else 0.0)
        fin[i] = start + service[i]
    return fin


def run_serving(args, spec, q):
    """Jobs arriving as a Poisson stream through the serving loop (lf_server:
    continuous batching, admission by memory budget, jobs side by side) against
    the same jobs one graph per call in arrival order (first come, first
    served on the same GPU): graphs/s over the stream and latency (arrival to
    result) percentiles."""
    import numpy as np
    import torch

    from paper_2210_03211_gb300 import build as lf_build
    from paper_2210_03211_gb300 import lazyfox
    from paper_2210_03211_gb300 import workloads as W

    rank, world, local = dist_setup(torch.cuda.is_available())
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU: the library has no CPU path")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        lf_build.build()
    barrier(world)
    lazyfox.load_library()
    graphs, arrivals = W.serving_jobs(args.jobs, seed=7 + rank, n_hi=args.max_nodes, rate=args.rate)
    J = len(graphs)
    thr, it = spec["threshold"], spec["max_iters"]
    # warm-up: two small jobs through both paths
    small = sorted(range(J), key=lambda i: graphs[i].src.shape[0])[:2]
    with lazyfox.Server(max_active=args.max_active) as srv:
        for i in small:
            srv.wait(srv.submit(graphs[i].src, graphs[i].dst, q, thr, it))
    for i in small:
        with lazyfox.Graph(graphs[i].src, graphs[i].dst) as g:
            g.run(q, thr, it)
            g.communities()
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks_s = ClockSampler("GPU-" + str(torch.cuda.get_device_properties(dev).uuid))
    clocks_s.start()
    # serving: submit at the arrival times
    with lazyfox.Server(max_active=args.max_active) as srv:
        t0 = time.perf_counter()
        ids = []
        for i in range(J):
            wait = arrivals[i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            ids.append(srv.submit(graphs[i].src, graphs[i].dst, q, thr, it))
        res = [srv.wait(j) for j in ids]
        served = {i: [c.tolist() for c in srv.community_list(ids[i])] for i in range(min(J, 16))}
    clocks = clocks_s.stop()
    lat_s = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in res])
    span_s = (max(r["t_done_ms"] for r in res) - min(r["t_submit_ms"] for r in res)) / 1e3
    # plain: one graph per call in arrival order; first come, first served
    service = np.zeros(J)
    same = True
    for i in range(J):
        torch.cuda.synchronize(dev)
        a = time.perf_counter()
        with lazyfox.Graph(graphs[i].src, graphs[i].dst) as g:
            g.run(q, thr, it)
            off, mem = g.communities()
            torch.cuda.synchronize(dev)
            service[i] = time.perf_counter() - a
            if i in served:
                same &= [mem[off[k]:off[k + 1]].tolist() for k in range(off.shape[0] - 1)] == served[i]
    fin = fifo_finish(arrivals, service)
    lat_p = (fin - arrivals) * 1e3
    span_p = fin[-1] - arrivals[0]
    value = J / span_s
    total_ms = reduce_max(span_s * 1e3, world, dev)
    if rank == 0:
        line = {
            "metric": METRIC, "value": reduce_sum(J, world, dev) / (total_ms / 1e3), "unit": "graphs/s",
            "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": total_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64", "data": "synthetic",
            "config": {"workload": spec["name"], "jobs": J, "rate_per_s": args.rate, "max_nodes": args.max_nodes,
                       "gain_rule": "literal (the library default, in the server and the plain calls)",
                       "edges": int(sum(g.src.shape[0] for g in graphs)), "queue_size": q, "threshold": thr,
                       "max_iters": it, "max_active": args.max_active, "parallelism": f"replicas x{world}",
                       "timed": "first arrival to last result; each job from host edge list to host communities"},
            "serving": {"graphs_per_s": value, "p50_ms": float(np.percentile(lat_s, 50)),
                        "p99_ms": float(np.percentile(lat_s, 99))},
            "plain": {"graphs_per_s": J / span_p, "p50_ms": float(np.percentile(lat_p, 50)),
                      "p99_ms": float(np.percentile(lat_p, 99)),
                      "timed": "one graph per call in arrival order, first come first served"},
            "speedup_vs_plain": value / (J / span_p),
            "results_equal_alone_and_served": bool(same),
            "clocks": clocks,
            "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": int(8 * sum(g.src.shape[0] for g in graphs)),
                    "d2h_bytes_per_step": None, "note": "jobs are host edge lists in and host communities out"},
        }
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    spec = WORKLOADS[args.workload]
    q = args.queue_size or spec["q"]
    if args.impl == "reference":
        return run_reference(args, spec, q)
    if args.workload == "batched":
        return run_batched(args, spec, q)
    if args.workload == "serving":
        return run_serving(args, spec, q)

    import numpy as np
    import torch

    from paper_2210_03211_gb300 import lazyfox
    from paper_2210_03211_gb300 import build as lf_build

    rank, world, local = dist_setup(torch.cuda.is_available())
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU: the library has no CPU path")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        lf_build.build()
    barrier(world)
    lazyfox.load_library()
    rule = args.gain_rule
    el = make_workload(spec)
    src_d = torch.from_numpy(el.src).to(dev)
    dst_d = torch.from_numpy(el.dst).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    # launch shape chosen once by the library's autotuner (two-iteration trials, untimed)
    with lazyfox.Graph(src_d, dst_d, stream=stream, gain_rule=rule) as g0:
        tune = g0.autotune(q, 2)
    shape = dict(warps_per_node=tune["warps_per_node"], warp_max_degree=tune["warp_max_degree"],
                 hub_degree=tune["hub_degree"])

    def one_step(s_d, d_d, queue, thr, iters, gain_rule, profile=False, use_graphs=True, shp=None):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = lazyfox.Graph(s_d, d_d, stream=stream, profile=profile, use_graphs=use_graphs, gain_rule=gain_rule,
                          **(shp or {}))
        st = g.run(queue, thr, iters)
        e1.record(stream)
        cs = g.create_stats()
        g.close()
        stream.synchronize()
        return e0.elapsed_time(e1), st, cs

    def step(profile=False, use_graphs=True):
        return one_step(src_d, dst_d, q, spec["threshold"], spec["max_iters"], rule, profile, use_graphs, shape)

    def timed(fn, steps, warmup, mark=False):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        barrier(world)
        torch.cuda.synchronize(dev)
        if mark:   # a profiler attached with --profile-from-start off sees the timed steps only
            torch.cuda.profiler.start()
        res = [fn() for _ in range(steps)]
        torch.cuda.synchronize(dev)
        if mark:
            torch.cuda.profiler.stop()
        barrier(world)
        return res

    gpu_id = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:  # noqa: BLE001 - older torch: fall back to the index
        pass
    sampler = ClockSampler(gpu_id)
    sampler.start()
    res = timed(step, args.steps, args.warmup, mark=True)
    clocks = sampler.stop()

    m = res[0][2]["num_edges"]
    local_units = sum(m * r[1].iterations for r in res)
    local_ms = sum(r[0] for r in res)
    total_ms = reduce_max(local_ms, world, dev)
    units = reduce_sum(local_units, world, dev)
    value = units / (total_ms / 1e3)
    step_s = local_ms / 1e3 / len(res)
    # triangle counting: merge-stream elements per second (a work rate, not
    # an HBM fraction: the kernels are issue-bound and re-read lists from L2)
    tri_gbs = statistics.median(r[2]["merge_bytes"] / (r[2]["ms_triangles"] / 1e3) / 1e9 for r in res
                                if r[2]["ms_triangles"] > 0) if m > 0 else 0.0
    launches = sum(r[2]["num_launches"] + r[1].num_launches for r in res)
    # the move evaluation's launch times come from profiled steps of the same
    # workload right after the timed region (profile mode records CUDA events
    # around each queue's evaluation launches and counts their algorithmic
    # bytes; it is kept out of the timed steps because the events and the byte
    # counter cost time)
    nprof = 1 if step_s > 5 else max(1, min(args.steps, 2))
    prof = [step(profile=True) for _ in range(nprof)]
    roofline_src = "profiled steps of the same workload right after the timed region"
    if any(math.isnan(r[1].prof_move_ms) for r in prof):
        prof = [step(profile=True, use_graphs=False) for _ in range(nprof)]
        roofline_src = "profiled steps with direct launches right after the timed region"
    persistent = rule == "meanfield" and q <= 256
    qpct = list(prof[-1][1].prof_queue_us) if persistent else None
    ev_bytes = sum(r[1].prof_move_bytes for r in prof)
    ev_ms = sum(r[1].prof_move_ms for r in prof)
    ev_launches = sum(r[1].prof_move_launches for r in prof)
    peak, peak_kind = measured_hbm()
    achieved = (ev_bytes / (ev_ms / 1e3) / 1e9) if ev_ms > 0 else 0.0
    if rule == "literal":
        kname = ("k_lit_eval + k_lit_big (move evaluation under the paper's gain; one launch = one queue's "
                 "evaluation kernels)")
        traffic = ncu_traffic("k_lit_eval", args.workload, q)
    else:
        kname = ("k_eval (move evaluation, one launch per queue)" if not persistent else
                 "k_iterate (persistent kernel: evaluate + apply of every queue, one launch per iteration)")
        traffic = ncu_traffic("k_eval", args.workload, q)
    roofline = {"kernel": kname, "bound": "hbm",
                "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": achieved / peak, "bytes_per_launch": ev_bytes / max(1, ev_launches),
                "mean_launch_us": 1e3 * ev_ms / max(1, ev_launches), "launches": ev_launches,
                "traffic": traffic["bytes_per_launch"] if traffic else None, "timed_in": roofline_src}
    if qpct:
        roofline["queue_us_p50_p90_p99_max"] = qpct

    secondary = []
    if not args.no_secondary:
        graphs = {args.workload: (src_d, dst_d)}
        for sec in spec.get("secondary", []):
            wl = sec["workload"]
            sspec = WORKLOADS[wl]
            if wl not in graphs:
                sel = make_workload(sspec)
                graphs[wl] = (torch.from_numpy(sel.src).to(dev), torch.from_numpy(sel.dst).to(dev))
            s_d, d_d = graphs[wl]
            fn = (lambda s_d=s_d, d_d=d_d, sec=sec, sspec=sspec:
                  one_step(s_d, d_d, sec["q"], sspec["threshold"], sspec["max_iters"], sec["rule"]))
            r2 = timed(fn, max(1, min(args.steps, 2)), 1)
            m2 = r2[0][2]["num_edges"]
            u2 = sum(m2 * r[1].iterations for r in r2)
            ms2 = reduce_max(sum(r[0] for r in r2), world, dev)
            secondary.append({"workload": sspec["name"], "queue_size": sec["q"], "gain_rule": sec["rule"],
                              "value": reduce_sum(u2, world, dev) / (ms2 / 1e3), "unit": UNIT,
                              "ms_per_step": ms2 / len(r2), "iterations": [r[1].iterations for r in r2]})
        del graphs

    e2e = None
    if not args.no_e2e:
        src_h = torch.from_numpy(el.src).pin_memory()
        dst_h = torch.from_numpy(el.dst).pin_memory()
        src_np, dst_np = src_h.numpy(), dst_h.numpy()
        e_units, e_secs, d2h = 0.0, 0.0, 0
        nsteps = 1 if step_s > 5 else max(1, min(args.steps, 3))
        for i in range(nsteps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            g = lazyfox.Graph(src_np, dst_np, gain_rule=rule, **shape)
            st = g.run(q, spec["threshold"], spec["max_iters"])
            off, mem = g.communities()
            t1 = time.perf_counter()
            g.close()
            if i == 0:
                continue   # first call pays one-time host setup; not timed
            e_units += g.m * st.iterations
            e_secs += t1 - t0
            d2h = off.nbytes + mem.nbytes + 48 * (st.iterations + 1)
        e_secs = reduce_max(e_secs, world, dev)
        e_units = reduce_sum(e_units, world, dev)
        e2e = {"value": e_units / e_secs, "unit": UNIT, "h2d_bytes_per_step": int(el.src.nbytes + el.dst.nbytes),
               "d2h_bytes_per_step": int(d2h), "steps": nsteps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cel, citers, what = cpu_sample_graph(spec)
        u, dt, it = time_oracle(cel, q, spec["threshold"], citers, rule)
        cpu = {"value": u / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{what} ({it} iteration(s), queue size {q}, gain rule {rule})",
               "seconds": dt, "host": host_info()}

    if rank == 0:
        r0 = res[0]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64", "data": "synthetic",
            "config": {"workload": spec["name"], "n": r0[2]["num_nodes"], "m": m, "queue_size": q,
                       "threshold": spec["threshold"], "max_iters": spec["max_iters"],
                       "gain_rule": rule + (" (the paper's: change of WCC-hat(P))" if rule == "literal" else
                                            " (departure: mean-field community score)"),
                       "iterations": [r[1].iterations for r in res], "parallelism": f"replicas x{world}",
                       "l2": "flushed before every step (256 MiB write); inputs resident in HBM"},
            "triangle_gbs": tri_gbs,
            "triangle_gbs_kind": ("work rate: merge-stream bytes (4 per list element streamed) per second of the "
                                  "triangle kernels; not DRAM traffic -- the kernels are issue-bound and re-read "
                                  "lists from L2 (ncu: DRAM at 10-12% of peak)"),
            "breakdown_ms": {"create": statistics.median(
                r[2]["ms_csr"] + r[2]["ms_orient"] + r[2]["ms_triangles"] + r[2]["ms_vt"] + r[2]["ms_order"]
                for r in res),
                "triangles": statistics.median(r[2]["ms_triangles"] for r in res),
                "init": statistics.median(r[1].ms_init for r in res),
                "iterations": statistics.median(r[1].ms_iterations for r in res),
                "queue_kernels_profiled": statistics.median(r[1].prof_move_ms for r in prof)},
            "roofline": roofline,
            "autotune": tune,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches,
        }
        if secondary:
            line["secondary"] = secondary
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
