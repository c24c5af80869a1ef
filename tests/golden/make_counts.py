"""Writes the oracle's embedding counts and result-set fingerprints for every
query of a workload to tests/golden/<workload>_counts.json.

Only the CPU oracle (plain backtracking, oracle/) and the seeded input
generator (synth/) run here; nothing of the CUDA library is imported.  The
full-size GPU parity tests compare every query's count and fingerprint with
this file.

    python tests/golden/make_counts.py medium
    python tests/golden/make_counts.py scale --max-bound 3e8

--max-bound skips queries whose admission bound (the spanning-tree
homomorphism count, an upper bound on the embeddings) exceeds the given
value; the file lists them as skipped, so a test knows which queries it
cannot check by count.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--max-bound", type=float, default=0.0, help="skip queries with a larger admission bound")
    ap.add_argument("--edge", action="store_true", help="count edge-isomorphic matches (Sec. VII-A)")
    args = ap.parse_args()
    w = synth.WORKLOADS[args.workload]
    g = synth.workload_graph(args.workload)
    qs = synth.queries(args.workload)
    O = oracle.OracleGraph.from_synth(g)
    count = oracle.count_edge if args.edge else oracle.count
    cmd = "python tests/golden/make_counts.py " + " ".join(sys.argv[1:])
    out = {"header": {"command": cmd,
                      "what": ("edge-isomorphic matches" if args.edge else "embeddings") +
                              " per query: exact count and the oracle fingerprint "
                              "(count, sum and xor of the chained row hashes) of the whole result set",
                      "workload": args.workload, "description": w.description,
                      "graph": {"kind": w.graph.kind, "n": w.graph.n, "m": w.graph.m, "seed": w.graph.seed},
                      "query_seed": w.query_seed, "queries": len(qs), "max_bound": args.max_bound or None,
                      "threads": oracle._threads()},
           "queries": []}
    t_all = time.perf_counter()
    for i, q in enumerate(qs):
        rec = {"index": i, "k": q.k, "edges": q.qm, "bound": q.bound}
        if args.max_bound and q.bound > args.max_bound:
            rec["skipped"] = "admission bound above --max-bound"
            out["queries"].append(rec)
            print(f"query {i}: skipped (bound {q.bound:.3g})", flush=True)
            continue
        t0 = time.perf_counter()
        c, fp = count(O, q)
        rec.update({"count": c, "fingerprint": [str(x) for x in fp], "seconds": round(time.perf_counter() - t0, 3)})
        out["queries"].append(rec)
        print(f"query {i}: k={q.k} count={c} in {rec['seconds']} s", flush=True)
    out["header"]["seconds"] = round(time.perf_counter() - t_all, 1)
    path = os.path.join(HERE, f"{args.workload}_counts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
