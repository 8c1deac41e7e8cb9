"""Writes tests/golden/oracle_counts.json. Calls only the CPU oracle and the input generators.

Run from the repository root: python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
import oracle  # noqa: E402


def main():
    out = {}
    g = inputs.workload_graph("er2000")
    gr, _ = oracle.relabel_by_degree(g)
    k, e = inputs.QUERIES["triangle"]
    out["er2000_triangle"] = oracle.count(gr, k, e, [(0, 1), (1, 2), (0, 2)])
    for name in ["k4", "c4", "house", "k5", "tailed_diamond_a"]:
        k, e = inputs.QUERIES[name]
        out[f"er2000_{name}"] = oracle.count(gr, k, e, oracle.symmetry_breaking_order(k, e))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(out)


if __name__ == "__main__":
    main()
