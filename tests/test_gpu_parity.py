"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact.

Inputs are seeded graphs from `inputs`; expected values come from `oracle` only.
"""
import itertools
from math import comb

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu
Q = inputs.QUERIES
MB = 1 << 20


def gload(huge, g, relabel=True):
    return huge.Graph(g.offsets, g.adj, flags=huge.RELABEL_BY_DEGREE if relabel else 0)


def oracle_graph(g, relabel=True):
    return oracle.relabel_by_degree(g)[0] if relabel else g


def test_closed_forms_complete_graphs(gpu_lib):
    huge = gpu_lib
    for n in (5, 9, 33):
        G = gload(huge, inputs.complete(n))
        for name, expect in [("triangle", comb(n, 3)), ("k4", comb(n, 4)), ("c4", 3 * comb(n, 4)),
                             ("house", 60 * comb(n, 5)), ("k5", comb(n, 5))]:
            k, e = Q[name]
            p = huge.Plan(G, k, e, order=oracle.connected_order(k, e))
            assert huge.enumerate(p) == expect, (n, name)


def test_complete_bipartite(gpu_lib):
    huge = gpu_lib
    G = gload(huge, inputs.complete_bipartite(7, 9))
    k, e = Q["c4"]
    assert huge.enumerate(huge.Plan(G, k, e, order=[0, 1, 3, 2])) == comb(7, 2) * comb(9, 2)
    k, e = Q["c6"]
    assert huge.enumerate(huge.Plan(G, k, e, order=[0, 1, 5, 2, 4, 3])) == 6 * comb(7, 3) * comb(9, 3)
    k, e = Q["triangle"]
    assert huge.enumerate(huge.Plan(G, k, e, order=[0, 1, 2])) == 0


def test_config_er2000_triangles(gpu_lib):
    """The K3 workload: ER n=2000, m=20000, partial order v0<v1<v2, count mode."""
    huge = gpu_lib
    g = inputs.workload_graph("er2000")
    gr = oracle_graph(g)
    k, e = Q["triangle"]
    po = [(0, 1), (1, 2), (0, 2)]
    expect = oracle.count(gr, k, e, po)
    G = gload(huge, g)
    for order in itertools.permutations(range(3)):
        assert huge.enumerate(huge.Plan(G, k, e, order=list(order), po=po)) == expect


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_graphs_named_queries_all_orders(gpu_lib, seed):
    huge = gpu_lib
    g = inputs.gnp(60, 1, 6, seed)
    gr = oracle_graph(g)
    G = gload(huge, g)
    for name in ["triangle", "k4", "c4", "house", "tailed_diamond_a", "diamond", "path4", "star4", "c5"]:
        k, e = Q[name]
        for po in (oracle.symmetry_breaking_order(k, e), []):
            expect = oracle.count(gr, k, e, po)
            orders = [o for o in itertools.permutations(range(k))
                      if all(any((o[j], o[t]) in set(map(tuple, e)) or (o[t], o[j]) in set(map(tuple, e))
                                 for t in range(j)) for j in range(1, k))]
            for o in orders[:: max(1, len(orders) // 6)]:
                got = huge.enumerate(huge.Plan(G, k, e, order=list(o), po=po))
                assert got == expect, (name, po, o)


def test_automatic_partial_order_matches_aut_invariant(gpu_lib):
    huge = gpu_lib
    g = inputs.gnp(40, 1, 4, 9)
    gr = oracle_graph(g)
    G = gload(huge, g)
    for s in range(12):
        k, e = inputs.random_query(3 + s % 4, 500 + s)
        aut = len(oracle.automorphisms(k, e))
        unbroken = oracle.count(gr, k, e, [])
        p = huge.Plan(G, k, e, order=oracle.connected_order(k, e))  # library's own partial order
        assert huge.enumerate(p) * aut == unbroken


def test_tree_verify_plans(gpu_lib):
    huge = gpu_lib
    g = inputs.gnp(50, 1, 5, 4)
    gr = oracle_graph(g)
    G = gload(huge, g)
    for name in ["k4", "c4", "house", "tailed_diamond_a", "k5"]:
        k, e = Q[name]
        po = oracle.symmetry_breaking_order(k, e)
        p = huge.Plan(G, k, e, order=oracle.connected_order(k, e), po=po, flags=huge.PLAN_TREE_VERIFY)
        ops = [s["op"] for s in p.describe()["chain"]["steps"]]
        if name != "path4":
            assert "VERIFY" in ops
        assert huge.enumerate(p) == oracle.count(gr, k, e, po), name


def test_tiny_level_capacity_forces_yield_and_resume(gpu_lib):
    """level_cap=32 makes every level yield and resume inside rows (Alg. 5 with Q_O tiny)."""
    huge = gpu_lib
    g = inputs.rmat(9, 8, 5)
    gr = oracle_graph(g)
    G = gload(huge, g)
    for name in ["triangle", "c4", "k4", "house", "k5"]:
        k, e = Q[name]
        po = oracle.symmetry_breaking_order(k, e)
        expect = oracle.count(gr, k, e, po)
        p = huge.Plan(G, k, e, order=oracle.connected_order(k, e), po=po)
        for cap in (32, 64, 4096):
            for fl in (0, huge.EF_NO_STEAL):
                assert huge.enumerate(p, level_cap=cap, flags=fl) == expect, (name, cap, fl)


def test_per_root_sample_parity_rmat(gpu_lib):
    """Sampled roots (hubs included) on R-MAT 13: per-root counts equal the oracle's."""
    huge = gpu_lib
    g = inputs.rmat(13, 8, 7)
    gr = oracle_graph(g)
    G = gload(huge, g)
    d = gr.degrees()
    roots = np.unique(np.concatenate([inputs.uniform(24, g.n, 3).astype(np.uint32),
                                      np.argsort(d)[-8:].astype(np.uint32)]))
    for name in ["k4", "c4", "tailed_diamond_a"]:
        k, e = Q[name]
        po = oracle.symmetry_breaking_order(k, e)
        order = oracle.connected_order(k, e)
        expect = oracle.count_roots(gr, k, e, roots, po, order)
        p = huge.Plan(G, k, e, order=order, po=po)
        for r, x in zip(roots, expect):
            assert huge.enumerate(p, roots=[r]) == x, (name, r)
        assert huge.enumerate(p, roots=roots) == int(expect.sum())


def test_level_rows_match_oracle_prefix_counts(gpu_lib):
    huge = gpu_lib
    g = inputs.rmat(9, 8, 8)
    gr = oracle_graph(g)
    G = gload(huge, g)
    for name in ["k4", "house", "c4"]:
        k, e = Q[name]
        po = oracle.symmetry_breaking_order(k, e)
        order = oracle.connected_order(k, e)
        p = huge.Plan(G, k, e, order=order, po=po)
        cnt, st = huge.enumerate(p, stats=True, flags=huge.EF_STATS)
        # prefix counts with the transitive closure of the partial order inside each prefix
        closure = set(po)
        changed = True
        while changed:
            changed = False
            for (a, b), (c, d2) in itertools.product(list(closure), list(closure)):
                if b == c and (a, d2) not in closure:
                    closure.add((a, d2))
                    changed = True
        pc = oracle.prefix_counts(gr, k, e, order, sorted(closure))
        assert st["level_rows"] == pc
        assert cnt == pc[-1]
        assert st["intersections"] == sum(pc[:-1])
        assert st["list_bytes"] > 0


def test_list_mode_multiset(gpu_lib):
    import torch

    huge = gpu_lib
    g = inputs.gnp(45, 1, 4, 12)
    gr = oracle_graph(g)
    G = gload(huge, g)
    for name in ["house", "tailed_diamond_a", "c4"]:
        k, e = Q[name]
        po = oracle.symmetry_breaking_order(k, e)
        expect = oracle.list_matches(gr, k, e, po)
        p = huge.Plan(G, k, e, order=oracle.connected_order(k, e)[::-1] if name == "c4" else
                      oracle.connected_order(k, e), po=po)
        sink = torch.zeros((len(expect) + 10, k), dtype=torch.int32, device="cuda")
        n = huge.enumerate(p, mode=huge.LIST, sink=sink)
        assert n == len(expect)
        rows = sink[:n].cpu().numpy().astype(np.uint32)
        rows = rows[np.lexsort(rows.T[::-1])]
        assert np.array_equal(rows, expect)


def test_list_mode_drain_small_sink(gpu_lib):
    """A sink smaller than the output: drained in pieces, the union equals the oracle's list."""
    import torch

    huge = gpu_lib
    g = inputs.gnp(40, 1, 3, 13)
    gr = oracle_graph(g)
    G = gload(huge, g)
    k, e = Q["c4"]
    po = oracle.symmetry_breaking_order(k, e)
    expect = oracle.list_matches(gr, k, e, po)
    assert len(expect) > 300
    sink = torch.zeros((257, k), dtype=torch.int32, device="cuda")
    got = []

    def drain(ptr, nrows):
        got.append(sink[:nrows].cpu().numpy().copy())

    p = huge.Plan(G, k, e, order=oracle.connected_order(k, e), po=po)
    n = huge.enumerate(p, mode=huge.LIST, sink=sink, drain=drain)
    assert n == len(expect)
    rows = np.concatenate(got).astype(np.uint32)
    rows = rows[np.lexsort(rows.T[::-1])]
    assert np.array_equal(rows, expect)
    with pytest.raises(huge.HugeError) as ei:
        huge.enumerate(p, mode=huge.LIST, sink=sink)
    assert ei.value.code == huge.ERANGE


def test_optimiser_plans_exact(gpu_lib):
    """Plans chosen by Alg. 1 (sampling estimator): EXTEND chains and PUSH-JOIN plans."""
    huge = gpu_lib
    g = inputs.rmat(9, 8, 21)
    gr = oracle_graph(g)
    G = gload(huge, g)
    for name in ["k4", "c4", "house", "path5", "tailed_diamond_a"]:
        k, e = Q[name]
        po = oracle.symmetry_breaking_order(k, e)
        expect = oracle.count(gr, k, e, po)
        for flags in (huge.PLAN_PLAIN, huge.PLAN_EXTEND_ONLY):
            p = huge.Plan(G, k, e, po=po, flags=flags)
            assert huge.enumerate(p) == expect, (name, flags, p.describe())
    g = inputs.er(3000, 12000, 22)
    gr = oracle_graph(g)
    G = gload(huge, g)
    k, e = Q["c6"]
    po = oracle.symmetry_breaking_order(k, e)
    p = huge.Plan(G, k, e, po=po)
    assert huge.enumerate(p) == oracle.count(gr, k, e, po), p.describe()


@pytest.mark.parametrize("name", ["c4", "path5", "c6", "path4"])
def test_push_join_plans(gpu_lib, name):
    huge = gpu_lib
    g = inputs.er(3000, 12000, 31) if name == "c6" else inputs.rmat(9, 8, 31)
    gr = oracle_graph(g)
    G = gload(huge, g)
    k, e = Q[name]
    po = oracle.symmetry_breaking_order(k, e)
    expect = oracle.count(gr, k, e, po)
    p = huge.Plan(G, k, e, po=po, flags=huge.PLAN_FORCE_JOIN)
    assert p.describe()["op"] == "PUSH-JOIN"
    assert huge.enumerate(p) == expect
    # a small memory bound forces partition passes of the join
    assert huge.enumerate(p, mem_bound=64 * MB) == expect


def test_push_join_list(gpu_lib):
    import torch

    huge = gpu_lib
    g = inputs.gnp(40, 1, 4, 17)
    gr = oracle_graph(g)
    G = gload(huge, g)
    k, e = Q["path5"]
    po = oracle.symmetry_breaking_order(k, e)
    expect = oracle.list_matches(gr, k, e, po)
    p = huge.Plan(G, k, e, po=po, flags=huge.PLAN_FORCE_JOIN)
    sink = torch.zeros((len(expect) + 5, k), dtype=torch.int32, device="cuda")
    n = huge.enumerate(p, mode=huge.LIST, sink=sink)
    assert n == len(expect)
    rows = sink[:n].cpu().numpy().astype(np.uint32)
    rows = rows[np.lexsort(rows.T[::-1])]
    assert np.array_equal(rows, expect)


def test_batch_random_queries(gpu_lib):
    huge = gpu_lib
    g = inputs.er(3000, 15000, 40)
    gr = oracle_graph(g)
    G = gload(huge, g)
    plans, expect = [], []
    for s in range(24):
        k, e = inputs.random_query(3 + s % 4, 40_000 + s)
        po = oracle.symmetry_breaking_order(k, e)
        plans.append(huge.Plan(G, k, e, order=oracle.connected_order(k, e), po=po))
        expect.append(oracle.count(gr, k, e, po))
    got = huge.enumerate_batch(plans)
    assert list(got) == expect
    cap, chunk = huge.autotune(plans, budget_ms=500)
    assert cap % 32 == 0
    assert list(huge.enumerate_batch(plans)) == expect


def test_edge_cases(gpu_lib):
    huge = gpu_lib
    # isolated vertices and an edgeless graph
    off = np.zeros(11, dtype=np.uint64)
    G = huge.Graph(off, np.zeros(0, dtype=np.uint32))
    k, e = Q["triangle"]
    assert huge.enumerate(huge.Plan(G, k, e, order=[0, 1, 2])) == 0
    # single-edge query: SCAN only
    g = inputs.er(100, 300, 3)
    G = gload(huge, g)
    assert huge.enumerate(huge.Plan(G, 2, [(0, 1)], order=[0, 1])) == 300
    assert huge.enumerate(huge.Plan(G, 2, [(0, 1)], order=[0, 1], po=[])) == 600
    # empty root range
    p = huge.Plan(G, 3, Q["triangle"][1], order=[0, 1, 2])
    assert huge.enumerate(p, root_range=(50, 50)) == 0
    # memory bound below the minimum
    with pytest.raises(huge.HugeError) as ei:
        huge.enumerate(p, mem_bound=1024)
    assert ei.value.code == huge.ENOMEM


def test_invalid_inputs_rejected(gpu_lib):
    huge = gpu_lib
    g = inputs.er(50, 100, 1)
    bad = g.adj.copy()
    bad[0], bad[1] = bad[1], bad[0]  # unsorted list
    with pytest.raises(huge.HugeError) as ei:
        huge.Graph(g.offsets, bad)
    assert ei.value.code == huge.EINVAL
    G = gload(huge, g)
    with pytest.raises(huge.HugeError):
        huge.Plan(G, 4, [(0, 1), (2, 3)])  # disconnected query
    with pytest.raises(huge.HugeError):
        huge.Plan(G, 3, Q["triangle"][1], po=[(0, 1), (1, 2), (2, 0)])  # cyclic PO
    with pytest.raises(huge.HugeError):
        huge.Plan(G, 4, Q["path4"][1], order=[0, 2, 1, 3])  # disconnected prefix


@pytest.mark.parametrize("relabel", [True, False])
def test_hub_bitmap_variant_every_vertex(gpu_lib, relabel):
    """Every vertex of degree >= 1 gets a bitmap, so every list check (EXTEND, the merge path's
    third lists, verify-only EXTEND) runs the bit probe; also the ragged small thresholds."""
    huge = gpu_lib
    g = inputs.rmat(10, 8, 41)
    gr = oracle_graph(g, relabel)
    G = gload(huge, g, relabel)
    names = ["triangle", "k4", "c4", "house", "tailed_diamond_a", "k5", "diamond"]
    want = {}
    for name in names:
        k, e = Q[name]
        want[name] = oracle.count(gr, k, e, oracle.symmetry_breaking_order(k, e))
    for min_deg in (1, 7, 40):
        G.set_hub_bitmaps(min_deg, 1 << 30)
        info = G.hub_info()
        assert info["count"] == int((gr.degrees() >= min_deg).sum())
        for name in names:
            k, e = Q[name]
            po = oracle.symmetry_breaking_order(k, e)
            expect = want[name]
            order = oracle.connected_order(k, e)
            assert huge.enumerate(huge.Plan(G, k, e, order=order, po=po)) == expect, (name, min_deg)
            assert huge.enumerate(huge.Plan(G, k, e, order=order, po=po), variant=1) == expect
            p = huge.Plan(G, k, e, order=order, po=po, flags=huge.PLAN_TREE_VERIFY)
            assert huge.enumerate(p) == expect, (name, "verify", min_deg)
    # a budget below one row keeps no bitmap
    G.set_hub_bitmaps(1, 16)
    assert G.hub_info()["count"] == 0


def test_hub_bitmap_budget_keeps_highest_degrees(gpu_lib):
    huge = gpu_lib
    g = inputs.rmat(12, 8, 42)
    gr = oracle_graph(g)
    G = gload(huge, g)
    blocks = (gr.n + 255) // 256  # a row: whole 256-bit blocks (32 bytes) plus a 4-byte rank entry each
    row = blocks * 36
    G.set_hub_bitmaps(2, 5 * row)
    info = G.hub_info()
    assert info["count"] == 5 and info["bytes"] == 5 * row + 4 * gr.n
    k, e = Q["c4"]
    po = oracle.symmetry_breaking_order(k, e)
    assert huge.enumerate(huge.Plan(G, k, e, po=po)) == oracle.count(gr, k, e, po)


def test_push_join_one_key_shared_by_many_rows(gpu_lib):
    """A star with 3000 leaves plus sparse leaf edges: the join key of the centre has a left
    group of thousands of rows, so one probe batch walks thousands of 32-candidate windows."""
    huge = gpu_lib
    from inputs import Graph

    n = 3001
    extra = inputs.er(n - 1, 4000, 51)
    es = {(0, v) for v in range(1, n)}
    src = np.repeat(np.arange(n - 1), extra.degrees())
    for u, v in zip(src, extra.adj.astype(np.int64)):
        if u < v:
            es.add((int(u) + 1, int(v) + 1))
    nbr = [[] for _ in range(n)]
    for u, v in es:
        nbr[u].append(v)
        nbr[v].append(u)
    off = np.concatenate([[0], np.cumsum([len(x) for x in nbr])]).astype(np.uint64)
    adj = np.concatenate([np.sort(np.asarray(x, dtype=np.uint32)) for x in nbr]).astype(np.uint32)
    g = Graph(off, adj, "star3000")
    gr = oracle_graph(g)
    G = gload(huge, g)
    for name in ["path4", "c4", "path5"]:
        k, e = Q[name]
        po = oracle.symmetry_breaking_order(k, e)
        p = huge.Plan(G, k, e, po=po, flags=huge.PLAN_FORCE_JOIN)
        assert p.describe()["op"] == "PUSH-JOIN"
        assert huge.enumerate(p) == oracle.count(gr, k, e, po), name


def test_torch_allocator_owns_library_buffers(gpu_lib):
    """With the binding's allocator hook, the graph's device buffers come from PyTorch's caching
    allocator (its allocated-bytes counter grows by at least the CSR) and go back on free."""
    import torch

    huge = gpu_lib
    huge.use_torch_allocator(True)
    g = inputs.rmat(14, 8, 61)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    G = gload(huge, g)
    held = torch.cuda.memory_allocated() - before
    assert held >= 4 * (g.n + 1) + 4 * g.nnz
    k, e = Q["triangle"]
    gr = oracle_graph(g)
    assert huge.enumerate(huge.Plan(G, k, e)) == oracle.count(gr, k, e, oracle.symmetry_breaking_order(k, e))
    G.free()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() <= before
    # back to cudaMalloc: nothing further shows up in torch's counter
    huge.use_torch_allocator(False)
    G2 = gload(huge, g)
    assert torch.cuda.memory_allocated() <= before
    G2.free()
    huge.use_torch_allocator(True)


def test_batch_per_plan_roots_caps_and_variants(gpu_lib):
    """huge_enumerate_batch_ex: every plan with its own root sample (hubs included, one plan
    with none), level capacity and intersection variant, all in one interleaved launch."""
    huge = gpu_lib
    g = inputs.er(3000, 15000, 45)  # random queries of up to 6 vertices: the oracle stays fast
    gr = oracle_graph(g)
    G = gload(huge, g)
    G.set_hub_bitmaps(14, 1 << 30)  # the highest-degree vertices get bitmaps too
    d = gr.degrees()
    plans, roots, caps, variants, expect = [], [], [], [], []
    for s in range(20):
        k, e = inputs.random_query(3 + s % 4, 45_000 + s)
        po = oracle.symmetry_breaking_order(k, e)
        order = oracle.connected_order(k, e)
        plans.append(huge.Plan(G, k, e, order=order, po=po))
        r = np.unique(np.concatenate([inputs.uniform(30 + s, g.n, 100 + s).astype(np.uint32),
                                      np.argsort(d)[-(1 + s % 5):].astype(np.uint32)]))
        if s == 7:
            r = r[:0]
        roots.append(r)
        caps.append([32, 64, 512, 2048][s % 4])
        variants.append([0, 1, 4][s % 3])
        expect.append(int(oracle.count_roots(gr, k, e, r, po, order).sum()) if len(r) else 0)
    got = huge.enumerate_batch(plans, roots=roots, level_caps=caps, variants=variants)
    assert list(got) == expect
    # the same plans over all roots, then one launch again: per-query counts are the oracle's
    full = [oracle.count(gr, p_k, p_e, oracle.symmetry_breaking_order(p_k, p_e))
            for p_k, p_e in (inputs.random_query(3 + s % 4, 45_000 + s) for s in range(20))]
    assert list(huge.enumerate_batch(plans, level_caps=caps)) == full
