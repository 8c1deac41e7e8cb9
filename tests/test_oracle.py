"""Pins for the CPU oracle: facts fixed by mathematics, not by the oracle's own code.

Each test would fail for a plausible mistake in the oracle: a dropped injectivity check
(closed forms on K_n, brute force), a dropped edge check (bipartite zero-triangle case, trace
identities), a wrong partial-order direction or index (|Aut| invariant with textbook group
orders), a wrong relabel (degree monotonicity, invariance), a wrong listing column order.
"""
import itertools
import json
import os
from math import comb

import numpy as np
import pytest

import inputs
import oracle

Q = inputs.QUERIES
HERE = os.path.dirname(os.path.abspath(__file__))

# |Aut(Q)| from the textbook structure of each query (not computed by the oracle).
AUT = {"triangle": 6, "k4": 24, "c4": 8, "k5": 120, "house": 2, "tailed_diamond_a": 2,
       "path3": 2, "path4": 2, "star4": 6, "c5": 10, "c6": 12, "diamond": 4,
       "tailed_triangle": 2}


def po_of(name):
    k, e = Q[name]
    return oracle.symmetry_breaking_order(k, e)


@pytest.mark.parametrize("name", sorted(AUT))
def test_automorphism_group_orders(name):
    k, e = Q[name]
    assert len(oracle.automorphisms(k, e)) == AUT[name]


@pytest.mark.parametrize("name", ["triangle", "k4", "c4", "k5", "house", "tailed_diamond_a",
                                  "path3", "star4", "c5", "diamond", "tailed_triangle"])
@pytest.mark.parametrize("n", [5, 6, 8])
def test_complete_graph_closed_form(name, n):
    """In K_n every injective map is a match, so #subgraphs = C(n,k) k! / |Aut(Q)|."""
    k, e = Q[name]
    g = inputs.complete(n)
    from math import factorial

    expect = comb(n, k) * factorial(k) // AUT[name]
    assert oracle.count(g, k, e, po_of(name)) == expect
    # without symmetry breaking every injective map counts: n!/(n-k)!
    assert oracle.count(g, k, e) == factorial(n) // factorial(n - k)


def test_named_closed_forms_on_kn():
    n = 9
    g = inputs.complete(n)
    assert oracle.count(g, 3, Q["triangle"][1], po_of("triangle")) == comb(n, 3)
    assert oracle.count(g, 4, Q["k4"][1], po_of("k4")) == comb(n, 4)
    assert oracle.count(g, 4, Q["c4"][1], po_of("c4")) == 3 * comb(n, 4)
    assert oracle.count(g, 5, Q["house"][1], po_of("house")) == 60 * comb(n, 5)


@pytest.mark.parametrize("a,b", [(2, 2), (3, 4), (5, 6), (7, 7)])
def test_complete_bipartite_cycles(a, b):
    """K_{a,b}: #C4 = C(a,2)C(b,2); #C6 = 6 C(a,3)C(b,3); no triangles, no odd cycles."""
    g = inputs.complete_bipartite(a, b)
    assert oracle.count(g, 4, Q["c4"][1], po_of("c4")) == comb(a, 2) * comb(b, 2)
    assert oracle.count(g, 6, Q["c6"][1], po_of("c6")) == 6 * comb(a, 3) * comb(b, 3)
    assert oracle.count(g, 3, Q["triangle"][1], po_of("triangle")) == 0
    assert oracle.count(g, 5, Q["c5"][1], po_of("c5")) == 0


def test_symmetry_breaking_orders_named():
    # K3: v0<v1<v2 as a chain of orbit representatives; C4 as derived from its dihedral group
    assert set(po_of("triangle")) == {(0, 1), (0, 2), (1, 2)}
    assert set(po_of("c4")) == {(0, 1), (0, 2), (0, 3), (1, 3)}


@pytest.mark.parametrize("seed", [11, 12, 13])
@pytest.mark.parametrize("name", ["triangle", "k4", "c4", "house", "tailed_diamond_a", "path4",
                                  "star4", "diamond"])
def test_brute_force_tiny(seed, name):
    k, e = Q[name]
    g = inputs.gnp(10, 1, 2, seed)
    po = po_of(name)
    assert oracle.count(g, k, e, po) == oracle.brute(g, k, e, po)
    assert oracle.count(g, k, e) == oracle.brute(g, k, e)


@pytest.mark.parametrize("seed", [21, 22])
def test_aut_invariant_and_order_invariance(seed):
    """count without PO == |Aut| * count with PO, for every connected matching order."""
    g = inputs.gnp(14, 2, 5, seed)
    for name in ["c4", "house", "tailed_diamond_a", "diamond", "k4", "path4"]:
        k, e = Q[name]
        po = po_of(name)
        base = oracle.count(g, k, e, po)
        assert oracle.count(g, k, e) == AUT[name] * base
        import itertools

        for order in itertools.permutations(range(k)):
            try:
                c = oracle.count(g, k, e, po, order=order)
            except ValueError:
                continue  # prefix not connected
            assert c == base


def test_random_queries_aut_invariant():
    g = inputs.gnp(12, 1, 2, 5)
    for s in range(20):
        k, e = inputs.random_query(3 + s % 3, 100 + s)
        po = oracle.symmetry_breaking_order(k, e)
        aut = len(oracle.automorphisms(k, e))
        assert oracle.count(g, k, e) == aut * oracle.count(g, k, e, po)
        assert oracle.count(g, k, e, po) == oracle.brute(g, k, e, po)


def _adj_matrix(g):
    a = np.zeros((g.n, g.n), dtype=np.float64)
    src = np.repeat(np.arange(g.n), g.degrees())
    a[src, g.adj.astype(np.int64)] = 1.0
    return a


def test_trace_identities_er():
    """#K3 = tr(A^3)/6 ; #C4 = (tr(A^4) - 2m - 4 sum_i C(d_i, 2)) / 8."""
    g = inputs.er(400, 3000, 7)
    a = _adj_matrix(g)
    a2 = a @ a
    t3 = np.trace(a2 @ a)
    t4 = np.trace(a2 @ a2)
    d = g.degrees()
    c4 = (t4 - 2 * g.m - 4 * np.sum(d * (d - 1) // 2)) / 8
    assert oracle.count(g, 3, Q["triangle"][1], po_of("triangle")) == round(t3 / 6)
    assert oracle.count(g, 4, Q["c4"][1], po_of("c4")) == round(c4)


def test_trace_identities_rmat_small():
    g = inputs.rmat(10, 8, 3)
    a = _adj_matrix(g)
    a2 = a @ a
    t3 = np.trace(a2 @ a)
    t4 = np.trace(a2 @ a2)
    d = g.degrees()
    c4 = (t4 - 2 * g.m - 4 * np.sum(d * (d - 1) // 2)) / 8
    gr, _ = oracle.relabel_by_degree(g)
    assert oracle.count(gr, 3, Q["triangle"][1], po_of("triangle")) == round(t3 / 6)
    assert oracle.count(gr, 4, Q["c4"][1], po_of("c4")) == round(c4)


def test_relabel_by_degree_properties():
    g = inputs.rmat(9, 8, 4)
    gr, new_of_old = oracle.relabel_by_degree(g)
    d_old, d_new = g.degrees(), gr.degrees()
    assert np.all(np.diff(d_new) >= 0)
    assert np.array_equal(d_new[new_of_old], d_old)
    # ties broken by original id
    old_of_new = np.argsort(new_of_old)
    for v in range(1, g.n):
        if d_new[v] == d_new[v - 1]:
            assert old_of_new[v] > old_of_new[v - 1]
    # lists sorted, symmetric
    for v in range(gr.n):
        lst = gr.adj[gr.offsets[v]:gr.offsets[v + 1]]
        assert np.all(np.diff(lst.astype(np.int64)) > 0)
    for name in ["triangle", "c4", "house"]:
        k, e = Q[name]
        assert oracle.count(g, k, e, po_of(name)) == oracle.count(gr, k, e, po_of(name))


def test_per_root_star_closed_form():
    """Star with 3 leaves, no PO, rooted at the centre: d(d-1)(d-2) matches per root."""
    g = inputs.rmat(9, 8, 6)
    k, e = Q["star4"]
    total, pr = oracle.count(g, k, e, order=[0, 1, 2, 3], per_root=True)
    d = g.degrees()
    assert np.array_equal(pr, d * (d - 1) * (d - 2))
    assert total == int(np.sum(d * (d - 1) * (d - 2)))


def test_listing_rows_are_matches():
    g = inputs.gnp(12, 1, 2, 9)
    for name in ["house", "c4", "tailed_diamond_a"]:
        k, e = Q[name]
        po = po_of(name)
        rows = oracle.list_matches(g, k, e, po)
        assert len(rows) == oracle.count(g, k, e, po)
        assert len({tuple(r) for r in rows}) == len(rows)
        es = set()
        for v in range(g.n):
            for w in g.adj[g.offsets[v]:g.offsets[v + 1]]:
                es.add((v, int(w)))
        for r in rows:
            assert len(set(r.tolist())) == k
            for u, v in e:
                assert (int(r[u]), int(r[v])) in es
            for a, b in po:
                assert r[a] < r[b]


def test_prefix_counts_closed_form():
    """On K_n the prefix q'_i of K4 is K_i: C(n, i) partial matches at every level."""
    n = 10
    g = inputs.complete(n)
    k, e = Q["k4"]
    assert oracle.prefix_counts(g, k, e, [0, 1, 2, 3], po_of("k4")) == [n, comb(n, 2), comb(n, 3),
                                                                       comb(n, 4)]


def test_prefix_counts_brute_force_on_a_sparse_graph():
    """Off the complete graph the prefix's own edges matter: every prefix count equals the brute
    force count of the sub-query induced by that prefix, with the partial-order pairs inside it
    (a dropped edge or a pair from outside the prefix changes some level)."""
    g = inputs.gnp(11, 1, 2, 23)
    for name, order in [("house", [0, 1, 4, 2, 3]), ("tailed_diamond_a", [4, 2, 0, 1, 3]),
                        ("c5", [0, 1, 2, 3, 4])]:
        k, e = Q[name]
        po = po_of(name)
        got = oracle.prefix_counts(g, k, e, order, po)
        assert got[0] == g.n
        for i in range(2, k + 1):
            idx = {v: j for j, v in enumerate(order[:i])}
            sub_e = [(idx[u], idx[v]) for u, v in e if u in idx and v in idx]
            sub_po = [(idx[a], idx[b]) for a, b in po if a in idx and b in idx]
            assert got[i - 1] == oracle.brute(g, i, sub_e, sub_po), (name, i)
        assert got[-1] == oracle.count(g, k, e, po)


def test_golden_config_er2000_triangles():
    """Stored value written by tests/golden/make_golden.py (calls only the oracle)."""
    with open(os.path.join(HERE, "golden", "oracle_counts.json")) as f:
        gold = json.load(f)
    g = inputs.workload_graph("er2000")
    gr, _ = oracle.relabel_by_degree(g)
    k, e = Q["triangle"]
    got = oracle.count(gr, k, e, [(0, 1), (1, 2), (0, 2)])
    assert got == gold["er2000_triangle"]
    # independent check: trace of A^3
    a = _adj_matrix(g)
    assert got == round(np.trace(a @ a @ a) / 6)
    # the G(n, m) expectation is a sanity range only: C(n,3) p^3 with p = m / C(n,2)
    p = 20000 / comb(2000, 2)
    assert 0.7 * comb(2000, 3) * p ** 3 < got < 1.3 * comb(2000, 3) * p ** 3


def test_stored_golden_values_are_the_oracles():
    """Every stored count the GPU is held to comes from the oracle: re-derive the ones that
    take seconds here (the G(n, m) workload's queries, the 1/64 Chung-Lu graph's 5-cliques and
    tailed diamonds, and R-MAT 20's 4-cycles from closed walks); the rest (R-MAT 20 triangles
    and 4-cliques, Chung-Lu 4M 5-cliques, the 1/64 graph's houses) take minutes each and are
    rewritten by tests/golden/make_golden.py."""
    with open(os.path.join(HERE, "golden", "oracle_counts.json")) as f:
        gold = json.load(f)
    g = oracle.relabel_by_degree(inputs.workload_graph("er2000"))[0]
    for name in ("triangle", "c4", "k4", "k5", "house", "tailed_diamond_a"):
        k, e = Q[name]
        assert oracle.count(g, k, e, po_of(name)) == gold["er2000_" + name], name
    h = inputs.workload_graph("chunglu64k")
    assert oracle.clique_count(h, 5) == gold["chunglu64k_k5"]
    k, e = Q["tailed_diamond_a"]
    hr = oracle.relabel_by_degree(h)[0]
    assert oracle.count(hr, k, e, po_of("tailed_diamond_a")) == gold["chunglu64k_tailed_diamond_a"]
    assert oracle.c4_count_trace(inputs.workload_graph("rmat20")) == gold["rmat20_c4"]


# ---- whole-graph counters that pin full-size workloads (no enumeration shared) ----

def test_walk_traces_match_dense_matrix_powers():
    """tr(A^3), tr(A^4) by sparse 2-walk counting equal numpy's dense matrix powers."""
    for g in [inputs.er(300, 2500, 3), inputs.rmat(9, 8, 5), inputs.complete_bipartite(4, 6)]:
        a = _adj_matrix(g)
        a2 = a @ a
        t3, t4 = oracle.walk_traces(g)
        assert t3 == round(np.trace(a2 @ a))
        assert t4 == round(np.trace(a2 @ a2))


@pytest.mark.parametrize("a,b", [(2, 2), (3, 5), (6, 6)])
def test_c4_trace_complete_bipartite(a, b):
    g = inputs.complete_bipartite(a, b)
    assert oracle.c4_count_trace(g) == comb(a, 2) * comb(b, 2)
    assert oracle.triangle_count_trace(g) == 0


@pytest.mark.parametrize("n", [4, 7, 10])
def test_trace_and_clique_counts_complete_graph(n):
    g = inputs.complete(n)
    assert oracle.c4_count_trace(g) == 3 * comb(n, 4)
    assert oracle.triangle_count_trace(g) == comb(n, 3)
    for k in range(1, 7):
        assert oracle.clique_count(g, k) == comb(n, k)


@pytest.mark.parametrize("seed", [31, 32])
def test_whole_graph_counters_agree_with_backtracker(seed):
    """The independent counters equal the backtracking oracle on mid-size power-law graphs."""
    g = inputs.rmat(11, 8, seed)
    assert oracle.c4_count_trace(g) == oracle.count(g, 4, Q["c4"][1], po_of("c4"))
    assert oracle.triangle_count_trace(g) == oracle.count(g, 3, Q["triangle"][1], po_of("triangle"))
    for name, k in [("triangle", 3), ("k4", 4), ("k5", 5)]:
        assert oracle.clique_count(g, k) == oracle.count(g, k, Q[name][1], po_of(name))
    assert oracle.clique_count(g, 2) == g.m


def test_clique_count_is_label_invariant():
    """The count does not depend on vertex ids (orientation ties are broken by id)."""
    g = inputs.rmat(10, 8, 9)
    gr, _ = oracle.relabel_by_degree(g)
    for k in (3, 4, 5):
        assert oracle.clique_count(g, k) == oracle.clique_count(gr, k)


# ---- labelled queries ----

def _two_label_complete(a, b):
    return inputs.complete(a + b), np.array([0] * a + [1] * b, dtype=np.uint32)


@pytest.mark.parametrize("a,b", [(3, 4), (5, 2), (6, 6)])
def test_labelled_triangles_in_two_coloured_complete_graph(a, b):
    """K_{a+b} with a vertices of label 0, b of label 1: #triangles labelled (0,0,1) = C(a,2) b,
    (0,1,1) = a C(b,2), (0,0,0) = C(a,3); ordered (no partial order): a(a-1) b for (0,0,1)."""
    g, dl = _two_label_complete(a, b)
    k, e = Q["triangle"]
    for ql, want in [((0, 0, 1), comb(a, 2) * b), ((0, 1, 1), a * comb(b, 2)), ((0, 0, 0), comb(a, 3)),
                     ((1, 1, 1), comb(b, 3))]:
        po = oracle.symmetry_breaking_order(k, e, ql)
        assert len(oracle.automorphisms(k, e, ql)) == (6 if len(set(ql)) == 1 else 2)
        assert oracle.count(g, k, e, po, dlabels=dl, qlabels=ql) == want, ql
    assert oracle.count(g, k, e, [], dlabels=dl, qlabels=(0, 0, 1)) == a * (a - 1) * b
    # a wildcard vertex takes either label
    any_ = oracle.ANY_LABEL
    assert oracle.count(g, k, e, [], dlabels=dl, qlabels=(0, any_, 1)) == a * b * (a + b - 2)


@pytest.mark.parametrize("seed", [61, 62])
def test_labelled_counts_partition_the_unlabelled_count(seed):
    """Every match has one tuple of image labels: summing the labelled counts (no partial order)
    over all query labellings gives the unlabelled count."""
    import itertools

    g = inputs.gnp(14, 1, 2, seed)
    dl = (inputs.uniform(g.n, 3, seed) % 3).astype(np.uint32)
    for name in ["triangle", "c4", "tailed_triangle", "path4"]:
        k, e = Q[name]
        total = sum(oracle.count(g, k, e, [], dlabels=dl, qlabels=ql)
                    for ql in itertools.product(range(3), repeat=k))
        assert total == oracle.count(g, k, e, [])


@pytest.mark.parametrize("seed", [71, 72, 73])
def test_labelled_brute_force_and_aut_invariant(seed):
    g = inputs.gnp(10, 1, 2, seed)
    dl = (inputs.uniform(g.n, 2, seed + 1) % 2).astype(np.uint32)
    for s in range(8):
        k, e = inputs.random_query(3 + s % 2, 300 + s)
        ql = tuple(int(x) for x in inputs.uniform(k, 2, 400 + s + seed) % 2)
        po = oracle.symmetry_breaking_order(k, e, ql)
        aut = len(oracle.automorphisms(k, e, ql))
        c = oracle.count(g, k, e, po, dlabels=dl, qlabels=ql)
        assert c == oracle.brute_labeled(g, k, e, dl, ql, po)
        assert oracle.count(g, k, e, [], dlabels=dl, qlabels=ql) == aut * c


# ---- directed queries ----

DIRECTED = {
    "cycle3": (3, [(0, 1), (1, 2), (2, 0)]),
    "transitive3": (3, [(0, 1), (1, 2), (0, 2)]),
    "path2": (3, [(0, 1), (1, 2)]),
    "out_star3": (4, [(0, 1), (0, 2), (0, 3)]),
    "cycle4": (4, [(0, 1), (1, 2), (2, 3), (3, 0)]),
    "bifan": (4, [(0, 2), (0, 3), (1, 2), (1, 3)]),
    "two_cycle_tail": (3, [(0, 1), (1, 0), (1, 2)]),
}
AUT_DIRECTED = {"cycle3": 3, "transitive3": 1, "path2": 1, "out_star3": 6, "cycle4": 4, "bifan": 4,
                "two_cycle_tail": 1}


def _complete_digraph(n):
    from inputs import Graph

    off = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.uint64)
    adj = np.array([v for u in range(n) for v in range(n) if v != u], dtype=np.uint32)
    return Graph(off, adj, f"DK{n}")


def _tournament(n):
    """Transitive tournament: arc i -> j iff i < j."""
    from inputs import Graph

    off = np.concatenate([[0], np.cumsum(np.arange(n - 1, -1, -1))]).astype(np.uint64)
    adj = np.array([v for u in range(n) for v in range(u + 1, n)], dtype=np.uint32)
    return Graph(off, adj, f"T{n}")


@pytest.mark.parametrize("name", sorted(DIRECTED))
def test_directed_automorphism_orders(name):
    k, a = DIRECTED[name]
    assert len(oracle.automorphisms(k, a, directed=True)) == AUT_DIRECTED[name]


@pytest.mark.parametrize("n", [5, 7])
def test_directed_closed_forms(n):
    """Complete digraph: every injective map matches, C(n,k) k!/|Aut|. Transitive tournament
    (arc i -> j iff i < j): no directed cycle or 2-cycle; C(n,3) transitive triangles and
    2-paths; C(n,4) out-stars (the smallest of 4 is the centre) and bifans (the 2 smallest are
    the sources)."""
    from math import factorial

    g = _complete_digraph(n)
    for name, (k, a) in DIRECTED.items():
        po = oracle.symmetry_breaking_order(k, a, directed=True)
        assert oracle.count_directed(g, k, a, po) == comb(n, k) * factorial(k) // AUT_DIRECTED[name], name
    t = _tournament(n)
    for name, want in [("cycle3", 0), ("transitive3", comb(n, 3)), ("path2", comb(n, 3)), ("cycle4", 0),
                       ("two_cycle_tail", 0), ("out_star3", comb(n, 4)), ("bifan", comb(n, 4))]:
        k, a = DIRECTED[name]
        assert oracle.count_directed(t, k, a, oracle.symmetry_breaking_order(k, a, directed=True)) == want, name


@pytest.mark.parametrize("seed", [81, 82])
def test_directed_brute_force_reversal_and_symmetric(seed):
    g = inputs.gnp_directed(9, 1, 3, seed)
    rg = oracle.reverse_csr(g)
    for name, (k, a) in DIRECTED.items():
        po = oracle.symmetry_breaking_order(k, a, directed=True)
        c = oracle.count_directed(g, k, a, po)
        assert c == oracle.brute_directed(g, k, a, po), name
        assert oracle.count_directed(g, k, a) == AUT_DIRECTED[name] * c
        # reversing every data arc and every query arc keeps the count
        assert oracle.count_directed(rg, k, [(y, x) for x, y in a], po) == c
    # an undirected graph seen as arcs both ways, a query with both arcs per edge: the
    # undirected count
    u = inputs.gnp(10, 1, 2, seed)
    for name in ("triangle", "c4", "tailed_triangle"):
        k, e = Q[name]
        both = e + [(y, x) for x, y in e]
        assert oracle.count_directed(u, k, both, po_of(name)) == oracle.count(u, k, e, po_of(name))


@pytest.mark.parametrize("seed", [91, 92])
def test_labelled_directed_brute_force_partition_and_aut(seed):
    """Labels and arcs together (Sec. 2 carries both over): the backtracker equals brute force;
    summed over every two-label labelling of the query, the counts give the unlabelled count;
    with the arc- and label-preserving symmetry-breaking order, count x |Aut| = the count with
    no order."""
    g = inputs.gnp_directed(9, 1, 3, seed)
    dl = (inputs.uniform(g.n, 2, seed) % 2).astype(np.uint32)
    for name, (k, a) in DIRECTED.items():
        total = 0
        for ql in itertools.product((0, 1), repeat=k):
            ql = list(ql)
            po = oracle.symmetry_breaking_order(k, a, ql, directed=True)
            c = oracle.count_directed(g, k, a, po, dlabels=dl, qlabels=ql)
            assert c == oracle.brute_directed(g, k, a, po, dlabels=dl, qlabels=ql), (name, ql)
            aut = len(oracle.automorphisms(k, a, ql, directed=True))
            free = oracle.count_directed(g, k, a, dlabels=dl, qlabels=ql)
            assert free == aut * c, (name, ql)
            total += free
        assert total == oracle.count_directed(g, k, a), name
        # a wildcard label matches everything
        any_l = [oracle.ANY_LABEL] * k
        assert oracle.count_directed(g, k, a, dlabels=dl, qlabels=any_l) == oracle.count_directed(g, k, a)


def test_labelled_directed_closed_form_on_a_two_coloured_complete_digraph():
    """Complete digraph with n0 vertices of label 0 and n1 of label 1: with no partial order every
    label-respecting injective map matches, n0^(c0) x n1^(c1) (falling factorials, c_L the
    query vertices of label L)."""
    from math import perm

    from inputs import Graph

    n0, n1 = 4, 5
    n = n0 + n1
    off = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.uint64)
    adj = np.array([v for u in range(n) for v in range(n) if v != u], dtype=np.uint32)
    g = Graph(off, adj, "DK9-2col")
    dl = np.array([0] * n0 + [1] * n1, dtype=np.uint32)
    for name, (k, a) in DIRECTED.items():
        for ql in ([0] * k, [1] * k, [i % 2 for i in range(k)]):
            c0, c1 = ql.count(0), ql.count(1)
            assert oracle.count_directed(g, k, a, dlabels=dl, qlabels=ql) == perm(n0, c0) * perm(n1, c1), (name, ql)


# --- Alg. 5 host model (oracle.scheduler) ---------------------------------------------------

def test_scheduler_model_reproduces_the_running_example():
    """Sec. 5.2's running example of the scheduler: queues of three batches, SCAN_1 fills its
    queue in slot 1 and yields; EXTEND_2, EXTEND_3 and SINK_4 follow; in slot 4 SINK_4 drains
    its input and the scheduler backtracks to EXTEND_3 (slot 5); after SINK_4 (slot 6)
    EXTEND_3 has no input, so control passes on to EXTEND_2 without a slot (slot 7). The
    figure with the batches is not in the text; a SCAN emitting one batch per source unit, an
    EXTEND_2 emitting two per batch and an EXTEND_3 emitting one reproduce every stated step."""
    from oracle import scheduler

    ops = [lambda u: ["s"], lambda b: ["x", "x"], lambda b: ["y"], lambda b: 1]
    res = scheduler.run(range(6), ops, cap=3)
    assert res["trace"][:7] == [0, 1, 2, 3, 2, 3, 1]
    # every source unit reaches the SINK: 6 units -> 12 batches at EXTEND_2 -> 12 at the SINK
    assert len(res["sink"]) == 12
    # SCAN stops at a full queue; EXTEND_2 overshoots by at most one batch's output
    assert res["peak"][0] == 3 and res["peak"][1] <= 3 - 1 + 2 and res["peak"][2] == 3


def test_scheduler_model_depth_first_at_capacity_one():
    """With room for one batch per queue the scheduler runs depth first: each source unit goes
    all the way to the SINK, and an empty EXTEND passes control back to SCAN without a slot."""
    from oracle import scheduler

    ops = [lambda u: ["a"], lambda b: ["b"], lambda b: 1]
    res = scheduler.run(range(3), ops, cap=1)
    assert res["trace"] == [0, 1, 2] * 3
    assert len(res["sink"]) == 3 and res["peak"] == [1, 1, 0]
    # an EXTEND that fans out 3:1 overfills its queue with its first batch, yields, and is
    # resumed once the SINK has drained it (backtracking)
    ops = [lambda u: ["a"], lambda b: ["b"] * 3, lambda b: 1]
    res = scheduler.run(range(2), ops, cap=2)
    assert res["trace"] == [0, 1, 2, 1, 2]
    assert len(res["sink"]) == 6 and res["peak"] == [2, 3, 0]
    with pytest.raises(ValueError):
        scheduler.run(range(3), ops, cap=0)


@pytest.mark.parametrize("name", ["triangle", "k4", "c4", "house", "tailed_diamond_a"])
def test_scheduler_model_counts_and_bounded_queues(name):
    """Alg. 5 over real partial matches: whatever the queue capacity and batch size, the SINK
    receives exactly the oracle's matches, and no queue holds more than cap - 1 batches plus one
    input batch's output. That output is at most batch_rows x D_G rows (Lemma 5.1), i.e. at
    most D_G batches."""
    from oracle import scheduler

    g = oracle.relabel_by_degree(inputs.gnp(40, 1, 4, 17))[0]
    off = np.asarray(g.offsets, dtype=np.int64)
    adj = [set(map(int, g.adj[off[u]:off[u + 1]])) for u in range(g.n)]
    dmax = int(np.diff(off).max())
    k, e = inputs.QUERIES[name]
    po = oracle.symmetry_breaking_order(k, e)
    order = oracle.connected_order(k, e)
    want = oracle.count(g, k, e, po)
    for cap in (1, 2, 5):
        for b in (1, 3, 16):
            source, ops = scheduler.extend_ops(adj, k, e, order, po, batch_rows=b)
            res = scheduler.run(source, ops, cap=cap)
            assert sum(res["sink"]) == want, (name, cap, b)
            assert all(p <= cap - 1 + max(dmax, 1) for p in res["peak"][:-1]), (name, cap, b, res["peak"])
