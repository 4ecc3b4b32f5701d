"""Command line: community detection on an edge-list file.

    python -m paper_2210_03211_gb300 EDGES [--queue-size Q] [--threshold T] [--max-iters N]
        [--output FILE] [--every-iteration DIR] [--resume COVER] [--ground-truth COVER] [--autotune]

EDGES is an undirected, unweighted edge list in the SNAP text format (two
non-negative integer ids per line, whitespace separated; lines starting with
'#' or '%' are comments; a '.gz' file is read compressed), the input the paper
describes (Methods, Input Data).  Communities are written one per line, member
ids separated by spaces (the format of SNAP's community files).  With
--every-iteration the communities after every iteration are saved as
DIR/iteration_<k>.txt (the per-iteration results the paper writes on
Friendster); --resume inserts a saved cover as the initial division (Methods,
Initial Clustering), so a run can continue from such a file; --ground-truth
reports the F1-score of the result against a reference cover (Methods,
Evaluation Criteria).  A JSON summary goes to standard output.  Every step runs
on the GPU through the library; this module only reads and writes files.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np


def read_edge_list(path: str):
    """(src, dst) int32 arrays of a SNAP-style edge list."""
    a = np.loadtxt(path, dtype=np.int64, comments=("#", "%"), usecols=(0, 1), ndmin=2)
    if a.size and (a.min() < 0 or a.max() > np.iinfo(np.int32).max):
        raise ValueError(f"{path}: node ids must lie in [0, 2^31 - 1]")
    return np.ascontiguousarray(a[:, 0], dtype=np.int32), np.ascontiguousarray(a[:, 1], dtype=np.int32)


def read_cover(path: str) -> list:
    """Communities of a cover file: one per line, ids separated by whitespace."""
    out = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line[0] in "#%":
                continue
            out.append(np.array([int(t) for t in line.split()], dtype=np.int32))
    return out


def write_cover(path: str, communities) -> None:
    with open(path, "w") as f:
        for c in communities:
            f.write(" ".join(str(int(v)) for v in c))
            f.write("\n")


def parse_args(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2210_03211_gb300",
                                 description="Fox / LazyFox overlapping community detection on one GPU")
    ap.add_argument("edges", help="edge list (SNAP text format, optionally .gz)")
    ap.add_argument("--queue-size", type=int, default=1, help="nodes evaluated against one snapshot (1 = Fox)")
    ap.add_argument("--threshold", type=float, default=0.01, help="relative WCC-hat change that stops the run")
    ap.add_argument("--max-iters", type=int, default=50)
    ap.add_argument("--output", help="file for the communities (default: none)")
    ap.add_argument("--every-iteration", metavar="DIR", help="save the communities after every iteration")
    ap.add_argument("--resume", metavar="COVER", help="start from this cover instead of the initial clustering")
    ap.add_argument("--ground-truth", metavar="COVER", help="report the F1-score against this cover")
    ap.add_argument("--autotune", action="store_true", help="choose the launch shape by timing short runs first")
    return ap.parse_args(argv)


def run(args, graph_cls=None, f1_fn=None, out=sys.stdout) -> dict:
    """The command on parsed arguments; graph_cls / f1_fn default to the
    library's Graph and cover_f1."""
    if graph_cls is None or f1_fn is None:
        from . import lazyfox
        graph_cls = graph_cls or lazyfox.Graph
        f1_fn = f1_fn or lazyfox.cover_f1
    src, dst = read_edge_list(args.edges)
    t0 = time.perf_counter()
    summary = {"edges_in": int(src.shape[0]), "queue_size": args.queue_size, "threshold": args.threshold}
    with graph_cls(src, dst) as g:
        summary.update(nodes=g.n, edges=g.m)
        if args.autotune:
            summary["autotune"] = g.autotune(args.queue_size, 1)
        if args.resume:
            g.set_partition(read_cover(args.resume))
        on_iteration = None
        if args.every_iteration:
            os.makedirs(args.every_iteration, exist_ok=True)

            def on_iteration(it, wcc):
                write_cover(os.path.join(args.every_iteration, f"iteration_{it}.txt"), g.community_list())
                return False
        st = g.run(args.queue_size, args.threshold, args.max_iters, on_iteration=on_iteration)
        communities = g.community_list()
    summary.update(iterations=st.iterations, converged=st.converged, wcc_initial=st.wcc_initial,
                   wcc=[float(v) for v in st.wcc_history], communities=len(communities),
                   memberships=int(sum(len(c) for c in communities)), seconds=time.perf_counter() - t0)
    if args.output:
        write_cover(args.output, communities)
    if args.ground_truth:
        summary["f1_vs_ground_truth"] = float(f1_fn(communities, read_cover(args.ground_truth))[0])
    out.write(json.dumps(summary) + "\n")
    return summary


def main(argv=None) -> int:
    run(parse_args(argv))
    return 0
