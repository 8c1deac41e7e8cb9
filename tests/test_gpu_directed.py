"""Directed queries on directed graphs on the GPU against the CPU oracle.

The library keeps every in-list after the out-lists and gives each EXTEND list a direction
bit; the oracle maps every query arc to a data arc by plain backtracking. Every form must give
the oracle's count: given orders, Alg. 1 plans (EXTEND chains and PUSH-JOIN), verify-only
chains, hub bitmaps on and off, 2-cycles in the query, labels together with directions.
"""
import itertools

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

DIRECTED = {
    "cycle3": (3, [(0, 1), (1, 2), (2, 0)]),
    "transitive3": (3, [(0, 1), (1, 2), (0, 2)]),
    "path2": (3, [(0, 1), (1, 2)]),
    "in_star3": (4, [(1, 0), (2, 0), (3, 0)]),
    "cycle4": (4, [(0, 1), (1, 2), (2, 3), (3, 0)]),
    "bifan": (4, [(0, 2), (0, 3), (1, 2), (1, 3)]),
    "two_cycle_tail": (3, [(0, 1), (1, 0), (1, 2)]),
    "feedback4": (4, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 1)]),
}


def _orders(k, arcs):
    es = {tuple(x) for x in arcs} | {(b, a) for a, b in arcs}
    return [o for o in itertools.permutations(range(k))
            if all(any((o[j], o[t]) in es for t in range(j)) for j in range(1, k))]


@pytest.mark.parametrize("seed", [1, 2])
def test_directed_queries_all_orders(gpu_lib, seed):
    huge = gpu_lib
    g = inputs.gnp_directed(60, 1, 6, seed)
    G = huge.Graph(g.offsets, g.adj, flags=huge.RELABEL_BY_DEGREE | huge.DIRECTED)
    for name, (k, a) in DIRECTED.items():
        po = oracle.symmetry_breaking_order(k, a, directed=True)
        want = oracle.count_directed(g, k, a, po)
        orders = _orders(k, a)
        for o in orders[:: max(1, len(orders) // 6)]:
            assert huge.enumerate(huge.Plan(G, k, a, order=list(o))) == want, (name, o)  # automatic partial order
        assert huge.enumerate(huge.Plan(G, k, a, order=list(orders[0]), po=[])) == oracle.count_directed(g, k, a)


def test_directed_planner_join_verify_hubs_and_labels(gpu_lib):
    huge = gpu_lib
    g = inputs.rmat_directed(11, 8, 7)
    G = huge.Graph(g.offsets, g.adj, flags=huge.RELABEL_BY_DEGREE | huge.DIRECTED)
    want = {}
    for name, (k, a) in DIRECTED.items():
        want[name] = oracle.count_directed(g, k, a, oracle.symmetry_breaking_order(k, a, directed=True))
    for hubs in (None, 0, 4):
        G.set_hub_bitmaps(hubs, 1 << 30)
        for name, (k, a) in DIRECTED.items():
            assert huge.enumerate(huge.Plan(G, k, a)) == want[name], (name, "alg1", hubs)
            p = huge.Plan(G, k, a, flags=huge.PLAN_TREE_VERIFY, order=oracle.connected_order(k, a))
            assert huge.enumerate(p) == want[name], (name, "verify", hubs)
        for name in ("cycle4", "bifan"):
            k, a = DIRECTED[name]
            pj = huge.Plan(G, k, a, flags=huge.PLAN_FORCE_JOIN)
            assert pj.describe()["op"] == "PUSH-JOIN"
            assert huge.enumerate(pj) == want[name], (name, "join", hubs)
    # directed and labelled together: oracle on both conditions via the partition identity
    dl = (inputs.uniform(g.n, 2, 5) % 2).astype(np.uint32)
    GL = huge.Graph(g.offsets, g.adj, flags=huge.RELABEL_BY_DEGREE | huge.DIRECTED, labels=dl)
    k, a = DIRECTED["transitive3"]
    total = sum(huge.enumerate(huge.Plan(GL, k, a, po=[], labels=list(ql), order=[0, 1, 2]))
                for ql in itertools.product(range(2), repeat=k))
    assert total == oracle.count_directed(g, k, a)


def test_directed_rejects_too_many_arcs_and_symmetric_equivalence(gpu_lib):
    huge = gpu_lib
    u = inputs.gnp(40, 1, 4, 3)
    # an undirected graph loaded as a directed one (every edge both ways), queries with both
    # arcs per edge: the undirected counts
    G = huge.Graph(u.offsets, u.adj, flags=huge.RELABEL_BY_DEGREE | huge.DIRECTED)
    Gu = huge.Graph(u.offsets, u.adj)
    for name in ("triangle", "c4", "tailed_triangle"):
        k, e = inputs.QUERIES[name]
        both = e + [(y, x) for x, y in e]
        assert huge.enumerate(huge.Plan(G, k, both)) == huge.enumerate(huge.Plan(Gu, k, e))
    # K5 with every arc both ways needs 8 lists at a vertex: rejected
    k, e = inputs.QUERIES["k5"]
    with pytest.raises(huge.HugeError):
        huge.Plan(G, k, e + [(y, x) for x, y in e])
