"""Digests of oracle runs on the 3.07M-node power-law workload, for the
full-size GPU parity test (tests/test_gpu_large_digests.py).

Calls only the oracle (oracle/) and the seeded workload generator: the
stored values never come from the CUDA path.  Per run (gain rule, queue
size, threshold -inf): cc and the node order (SHA-256 of the int32 array),
and after each recorded iteration the WCC-hat total (as a hex float), joins,
leaves and the SHA-256 of the membership CSR (int64 offsets over dense ids,
then int32 community ids).  The paper's gain costs the oracle a pass over
each candidate community (hours per iteration on this graph), so its runs
are recorded after iteration 1; the mean-field runs after iterations 1, 2
and 20.

    python tests/golden/make_large_digests.py [--rule literal|meanfield] [--out FILE]

Runs the (rule, queue size) jobs in parallel, one process each, and rewrites
the output (default tests/golden/large_digests_<rule>.json) as each job
finishes; hours of CPU time.
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

JOBS = {"literal": [("literal", 65536, [1]), ("literal", 1024, [1])],
        "meanfield": [("meanfield", 65536, [1, 2, 20]), ("meanfield", 1024, [1, 2, 20])]}


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(a.tobytes())
    return h.hexdigest()


def job(spec):
    import numpy as np

    import oracle
    from paper_2210_03211_gb300 import workloads as W
    rule, q, points = spec
    t0 = time.time()
    el = W.large_like()
    g = oracle.OracleGraph(el.src, el.dst)
    out = dict(rule=rule, queue_size=q, n=g.n, m=g.m, cc=float(g.cc).hex(),
               order_sha256=sha(np.ascontiguousarray(g.order(), dtype=np.int32)), points=[])
    for it in points:
        r = g.run(q, -float("inf"), it, rule=rule)
        s = g.state()
        out["points"].append(dict(iteration=it, T=[float(v).hex() for v in r["T"]],
                                  joins=[int(v) for v in r["joins"]], leaves=[int(v) for v in r["leaves"]],
                                  T0=float(r["T0"]).hex(),
                                  memberships_sha256=sha(np.ascontiguousarray(s["mem_off"], dtype=np.int64),
                                                         np.ascontiguousarray(s["mem_ids"], dtype=np.int32)),
                                  memberships=int(s["mem_off"][-1])))
        print(f"{rule} q={q} iteration {it} done after {time.time() - t0:.0f} s", flush=True)
    out["cpu_seconds"] = time.time() - t0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rule", choices=sorted(JOBS), required=True)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    out = args.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"large_digests_{args.rule}.json")
    jobs = JOBS[args.rule]
    res = []
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        for r in pool.imap_unordered(job, jobs):
            res.append(r)
            res.sort(key=lambda x: -x["queue_size"])
            doc = dict(workload="large_like() -- 3.07M nodes, power law (gamma 2.2), seed 4", threshold="-inf",
                       written_by="tests/golden/make_large_digests.py (oracle only)", runs=res)
            with open(out, "w") as f:
                json.dump(doc, f, indent=1)
            print("wrote", out, "with", len(res), "run(s)", flush=True)


if __name__ == "__main__":
    main()
