"""Writes tests/golden/oracle_counts.json. Calls only the CPU oracle and the input generators.

Run from the repository root: python tests/golden/make_golden.py [--small]

Stored values:
* er2000_*: the K3 workload's graph (G(n=2000, m=20000)), backtracking oracle.
* rmat20_*: the whole R-MAT scale-20 workload. 4-cycles from the closed-walk identity
  tr(A^4) = 8 #C4 + 2m + 4 sum C(d, 2); 4-cliques and triangles from the degree-orientation
  clique counter. Neither enumerates matches the way the backtracker or the library does.
* chunglu4m_k5: 5-cliques of the whole Chung-Lu 4M workload (clique counter).
* chunglu64k_*: the Chung-Lu recipe at 1/64 scale, whole graph, backtracking oracle (hubs
  included); K5 also cross-checked with the clique counter.
--small recomputes only the er2000 entries and keeps the stored large ones.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
import oracle  # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts.json")


def po(name):
    k, e = inputs.QUERIES[name]
    return oracle.symmetry_breaking_order(k, e)


def main():
    try:
        with open(PATH) as f:
            out = json.load(f)
    except OSError:
        out = {}
    g = inputs.workload_graph("er2000")
    gr, _ = oracle.relabel_by_degree(g)
    k, e = inputs.QUERIES["triangle"]
    out["er2000_triangle"] = oracle.count(gr, k, e, [(0, 1), (1, 2), (0, 2)])
    for name in ["k4", "c4", "house", "k5", "tailed_diamond_a"]:
        k, e = inputs.QUERIES[name]
        out[f"er2000_{name}"] = oracle.count(gr, k, e, po(name))
    if "--small" not in sys.argv:
        t = time.time()
        g = inputs.workload_graph("rmat20")
        out["rmat20_c4"] = oracle.c4_count_trace(g)
        out["rmat20_triangle"] = oracle.triangle_count_trace(g)
        assert oracle.clique_count(g, 3) == out["rmat20_triangle"]
        out["rmat20_k4"] = oracle.clique_count(g, 4)
        print("rmat20", time.time() - t, flush=True)
        g = inputs.workload_graph("chunglu4m")
        out["chunglu4m_k5"] = oracle.clique_count(g, 5)
        print("chunglu4m", time.time() - t, flush=True)
        g = inputs.workload_graph("chunglu64k")
        gr, _ = oracle.relabel_by_degree(g)
        for name in ["k5", "tailed_diamond_a", "house"]:
            k, e = inputs.QUERIES[name]
            out[f"chunglu64k_{name}"] = oracle.count(gr, k, e, po(name))
            print(name, time.time() - t, flush=True)
        assert oracle.clique_count(g, 5) == out["chunglu64k_k5"]
    with open(PATH, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(out)


if __name__ == "__main__":
    main()
