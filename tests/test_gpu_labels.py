"""Labelled queries on the GPU against the CPU oracle (Sec. 2: labels carry over to the method).

The library groups the data graph's ids by label, so a labelled query vertex becomes an id-range
bound; the oracle checks label(f(v)) = label(v) per assignment. Every form must give the
oracle's count: given orders, Alg. 1 plans (EXTEND chains and PUSH-JOIN), verify-only EXTEND
chains, hub bitmaps on and off, LIST rows, batched launches, wildcard labels and a label the
graph does not have.
"""
import itertools

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu
Q = inputs.QUERIES
ANY = oracle.ANY_LABEL


def _labels(n, nl, seed):
    return (inputs.uniform(n, nl, seed) % nl).astype(np.uint32)


def _orders(k, e):
    es = {tuple(x) for x in e} | {(b, a) for a, b in e}
    return [o for o in itertools.permutations(range(k))
            if all(any((o[j], o[t]) in es for t in range(j)) for j in range(1, k))]


@pytest.mark.parametrize("seed", [1, 2])
def test_labelled_named_queries_all_orders(gpu_lib, seed):
    huge = gpu_lib
    g = inputs.gnp(70, 1, 5, seed)
    dl = _labels(g.n, 3, 10 + seed)
    G = huge.Graph(g.offsets, g.adj, labels=dl, nlabels=3)
    rng = np.random.default_rng(seed)
    for name in ["triangle", "k4", "c4", "house", "tailed_diamond_a", "diamond", "path4", "star4"]:
        k, e = Q[name]
        for trial in range(3):
            ql = [int(x) for x in rng.integers(0, 3, k)]
            if trial == 2:
                ql[int(rng.integers(k))] = ANY
            po = oracle.symmetry_breaking_order(k, e, ql)
            want = oracle.count(g, k, e, po, dlabels=dl, qlabels=ql)
            orders = _orders(k, e)
            for o in orders[:: max(1, len(orders) // 5)]:
                got = huge.enumerate(huge.Plan(G, k, e, order=list(o), labels=ql))  # automatic partial order
                assert got == want, (name, ql, o)
            assert huge.enumerate(huge.Plan(G, k, e, order=list(orders[0]), po=po, labels=ql)) == want
            assert huge.enumerate(huge.Plan(G, k, e, order=list(orders[0]), po=[], labels=ql)) == \
                oracle.count(g, k, e, [], dlabels=dl, qlabels=ql)


def test_labelled_planner_join_verify_and_hubs(gpu_lib):
    huge = gpu_lib
    g = inputs.rmat(11, 8, 5)
    dl = _labels(g.n, 2, 77)
    G = huge.Graph(g.offsets, g.adj, labels=dl)
    cases = [("c4", [0, 1, 0, 1]), ("k4", [0, 0, 1, 1]), ("path5", [1, 0, ANY, 0, 1]),
             ("tailed_diamond_a", [0, 0, 1, 1, 0]), ("triangle", [1, 1, 1])]
    wants = {}
    for name, ql in cases:
        k, e = Q[name]
        wants[name] = oracle.count(g, k, e, oracle.symmetry_breaking_order(k, e, ql), dlabels=dl, qlabels=ql)
    for hubs in (None, 0, 8):
        G.set_hub_bitmaps(hubs, 1 << 30)
        for name, ql in cases:
            k, e = Q[name]
            want = wants[name]
            assert huge.enumerate(huge.Plan(G, k, e, labels=ql)) == want, (name, "alg1", hubs)
            p = huge.Plan(G, k, e, labels=ql, flags=huge.PLAN_TREE_VERIFY, order=oracle.connected_order(k, e))
            assert huge.enumerate(p) == want, (name, "verify", hubs)
            if name in ("c4", "path5"):
                pj = huge.Plan(G, k, e, labels=ql, flags=huge.PLAN_FORCE_JOIN)
                assert pj.describe()["op"] == "PUSH-JOIN"
                assert huge.enumerate(pj) == want, (name, "join", hubs)


def test_labelled_list_rows_batch_and_missing_label(gpu_lib):
    import torch

    huge = gpu_lib
    g = inputs.gnp(60, 1, 4, 9)
    dl = _labels(g.n, 3, 19)
    G = huge.Graph(g.offsets, g.adj, labels=dl, nlabels=4)  # label 3 has no vertex
    new = G.new_ids()
    ls = G.label_ranges()
    assert len(ls) == 5 and ls[3] == ls[4] == g.n
    assert np.all(np.diff(ls) == np.bincount(dl, minlength=4))
    # every vertex's new id lies in its label's range
    assert np.all((new >= ls[dl]) & (new < ls[dl + 1]))
    k, e = Q["house"]
    ql = [0, 1, 2, 0, ANY]
    po = oracle.symmetry_breaking_order(k, e, ql)
    want = oracle.count(g, k, e, po, dlabels=dl, qlabels=ql)
    p = huge.Plan(G, k, e, labels=ql, order=oracle.connected_order(k, e))
    sink = torch.zeros((want + 8, k), dtype=torch.int32, device="cuda")
    n = huge.enumerate(p, mode=huge.LIST, sink=sink)
    assert n == want
    rows = sink[:n].cpu().numpy().astype(np.int64)
    old_of_new = np.argsort(new)
    lab_new = dl[old_of_new]
    for v, L in enumerate(ql):
        if L != ANY:
            assert np.all(lab_new[rows[:, v]] == L)
    assert len({tuple(r) for r in rows}) == n
    # a label no vertex carries: no match
    assert huge.enumerate(huge.Plan(G, 3, Q["triangle"][1], labels=[3, 0, 0])) == 0
    # batched labelled plans
    plans, expect = [], []
    for s in range(10):
        kk, ee = inputs.random_query(3 + s % 3, 700 + s)
        qq = [int(x) for x in _labels(kk, 3, 800 + s)]
        plans.append(huge.Plan(G, kk, ee, labels=qq, order=oracle.connected_order(kk, ee)))
        expect.append(oracle.count(g, kk, ee, oracle.symmetry_breaking_order(kk, ee, qq), dlabels=dl, qlabels=qq))
    assert list(huge.enumerate_batch(plans)) == expect
    # query labels on an unlabelled graph are rejected
    G2 = huge.Graph(g.offsets, g.adj)
    with pytest.raises(huge.HugeError):
        huge.Plan(G2, 3, Q["triangle"][1], labels=[0, 0, 0])


def test_labelled_rmat_whole_graph(gpu_lib):
    """R-MAT 13 with 4 labels, default hub bitmaps, Alg. 1 plans, every root."""
    huge = gpu_lib
    g = inputs.rmat(13, 8, 23)
    dl = _labels(g.n, 4, 29)
    G = huge.Graph(g.offsets, g.adj, labels=dl)
    for name, ql in [("k4", [0, 1, 1, 2]), ("c4", [3, 3, 3, 3]), ("house", [0, 1, 2, 3, 0])]:
        k, e = Q[name]
        po = oracle.symmetry_breaking_order(k, e, ql)
        assert huge.enumerate(huge.Plan(G, k, e, labels=ql)) == oracle.count(g, k, e, po, dlabels=dl, qlabels=ql)
