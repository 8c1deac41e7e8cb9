"""Whole-graph parity at full size: the launch the benchmark times, on the whole workload,
against stored values written by tests/golden/make_golden.py (which calls only the oracle):
the closed-walk identity for 4-cycles, the degree-orientation clique counter for cliques, and
the backtracking oracle for the 5-vertex queries on the 1/64-scale Chung-Lu graph (hubs
included). Every intersection variant (hub bitmaps on or off, merge path on or off) must give
the same exact count."""
import json
import os

import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
MEM_BOUND = 8 << 30


def golden():
    with open(os.path.join(HERE, "golden", "oracle_counts.json")) as f:
        return json.load(f)


def test_rmat20_whole_graph_counts_match_golden(gpu_lib):
    """The benchmark step: Alg. 1 plans for the 4-clique and the 4-cycle over every root."""
    huge = gpu_lib
    gold = golden()
    g = inputs.workload_graph("rmat20")
    G = huge.Graph(g.offsets, g.adj)
    assert G.hub_info()["count"] > 0  # the default degree buckets give the hubs bitmaps
    for name in ("k4", "c4"):
        k, e = inputs.QUERIES[name]
        p = huge.Plan(G, k, e)
        assert huge.enumerate(p, mem_bound=MEM_BOUND) == gold[f"rmat20_{name}"], name


def test_rmat20_counts_identical_across_intersection_variants(gpu_lib):
    """Hub bitmaps off / default / many, merge path off / on: the same exact counts."""
    huge = gpu_lib
    gold = golden()
    g = inputs.workload_graph("rmat20")
    G = huge.Graph(g.offsets, g.adj)
    k, e = inputs.QUERIES["k4"]
    p = huge.Plan(G, k, e, order=[0, 3, 2, 1])
    for min_deg, max_bytes in ((0, 0), (64, 2 << 30), (None, 1 << 30)):
        G.set_hub_bitmaps(min_deg, max_bytes)
        for variant in (1, 8):
            assert huge.enumerate(p, mem_bound=MEM_BOUND, variant=variant) == gold["rmat20_k4"], (min_deg, variant)


def test_rmat20_triangles_match_trace(gpu_lib):
    huge = gpu_lib
    g = inputs.workload_graph("rmat20")
    G = huge.Graph(g.offsets, g.adj)
    k, e = inputs.QUERIES["triangle"]
    assert huge.enumerate(huge.Plan(G, k, e), mem_bound=MEM_BOUND) == golden()["rmat20_triangle"]


def test_chunglu64k_whole_graph_5vertex_queries(gpu_lib):
    """The Chung-Lu recipe at 1/64 scale, every root (hubs included): K5, house and tailed
    diamond with Alg. 1's plans and with hub bitmaps off."""
    huge = gpu_lib
    gold = golden()
    g = inputs.workload_graph("chunglu64k")
    G = huge.Graph(g.offsets, g.adj)
    for hubs in (True, False):
        G.set_hub_bitmaps(None if hubs else 0)
        for name in ("k5", "house", "tailed_diamond_a"):
            k, e = inputs.QUERIES[name]
            po = oracle.symmetry_breaking_order(k, e)
            p = huge.Plan(G, k, e, po=po)
            assert huge.enumerate(p, mem_bound=MEM_BOUND) == gold[f"chunglu64k_{name}"], (name, hubs)


def test_chunglu4m_whole_graph_k5(gpu_lib):
    huge = gpu_lib
    g = inputs.workload_graph("chunglu4m")
    G = huge.Graph(g.offsets, g.adj)
    k, e = inputs.QUERIES["k5"]
    assert huge.enumerate(huge.Plan(G, k, e), mem_bound=MEM_BOUND) == golden()["chunglu4m_k5"]
