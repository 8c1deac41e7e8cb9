"""The planner on the host (huge_plan_offline, no GPU): compiled plans run by a plain Python
interpreter of their operators give the oracle's counts and matches, and Alg. 1's dynamic
programme finds the cheapest plan an exhaustive search over all plans finds.

The interpreter reads each operator as its descriptor states it (Sec. 4.2): an EXTEND binds
the new vertex to the common neighbours of the rows' `ext` positions, above every `lo` and below
every `hi` position (strict), and distinct from every `inj` position; a VERIFY (Sec. 5.2) keeps
a row iff each `ext` position is adjacent to its `with` position; a PUSH-JOIN joins the two
sides' rows on equal keys, then requires distinct non-key vertices across the sides and the
cross-side partial-order pairs. Expected values come from `oracle` only.
"""
import functools
import itertools

import numpy as np
import pytest

import inputs
import oracle
from paper_2103_14294_b300 import huge

Q = inputs.QUERIES


def _adj_sets(g):
    off = np.asarray(g.offsets, dtype=np.int64)
    return [set(map(int, g.adj[off[u]:off[u + 1]])) for u in range(len(off) - 1)]


def run_chain(adj, chain):
    """Rows (in matching-order positions) produced by the chain's operators from every root."""
    rows = [(r,) for r in range(len(adj))]
    for st in chain["steps"]:
        out = []
        if st["op"] == "EXTEND":
            for f in rows:
                cand = set.intersection(*[adj[f[p]] for p in st["ext"]])
                for u in cand:
                    if all(u > f[p] for p in st["lo"]) and all(u < f[p] for p in st["hi"]) and \
                            all(u != f[p] for p in st["inj"]):
                        out.append(f + (u,))
        else:
            assert st["op"] == "VERIFY"
            out = [f for f in rows if all(f[b] in adj[f[a]] for a, b in zip(st["ext"], st["with"]))]
        rows = out
    return rows


def to_query_order(rows, order):
    """Rows in matching-order positions -> rows indexed by query vertex."""
    res = np.zeros((len(rows), len(order)), dtype=np.int64)
    for i, f in enumerate(rows):
        for p, v in enumerate(order):
            res[i, v] = f[p]
    return res


def run_join(adj, plan):
    js = plan["join_spec"]
    left = to_query_order(run_chain(adj, plan["left"]), plan["left"]["order"])
    right = to_query_order(run_chain(adj, plan["right"]), plan["right"]["order"])
    index = {}
    for R in right:
        index.setdefault(tuple(int(R[c]) for c in js["rkey"]), []).append(R)
    out = []
    for L in left:
        for R in index.get(tuple(int(L[c]) for c in js["lkey"]), []):
            if any(L[a] == R[b] for a in js["nonkey_l"] for b in js["nonkey_r"]):
                continue
            if not all(L[a] < R[b] for a, b in zip(js["lr_l"], js["lr_r"])):
                continue
            if not all(R[b] < L[a] for b, a in zip(js["rl_r"], js["rl_l"])):
                continue
            row = np.zeros(plan["k"], dtype=np.int64)
            for c, col in enumerate(js["out_col_l"]):
                row[col] = L[c]
            for c, col in enumerate(js["out_col_r"]):
                if col >= 0:
                    row[col] = R[c]
            out.append(row)
    return np.asarray(out, dtype=np.int64).reshape(-1, plan["k"])


def _sorted_rows(a):
    a = np.asarray(a, dtype=np.int64)
    return a[np.lexsort(a.T[::-1])] if len(a) else a


def connected_orders(k, edges):
    es = {frozenset(e) for e in map(tuple, edges)}
    for o in itertools.permutations(range(k)):
        if all(any(frozenset((o[j], o[t])) in es for t in range(j)) for j in range(1, k)):
            yield list(o)


@pytest.mark.parametrize("seed", [1, 2])
def test_chain_plans_of_every_order_match_oracle(seed):
    g = oracle.relabel_by_degree(inputs.gnp(24, 1, 4, 70 + seed))[0]
    adj = _adj_sets(g)
    for name in ["triangle", "k4", "c4", "diamond", "tailed_triangle", "house", "tailed_diamond_a", "c5",
                 "path4", "star4"]:
        k, e = Q[name]
        po = oracle.symmetry_breaking_order(k, e)
        want = oracle.count(g, k, e, po)
        orders = list(connected_orders(k, e))
        for o in orders[:: max(1, len(orders) // 8)]:
            for fl in (huge.PLAN_PLAIN, huge.PLAN_TREE_VERIFY):
                plan = huge.plan_offline(k, e, order=o, po=po, flags=fl)
                assert plan["op"] == "EXTEND-CHAIN" and plan["chain"]["order"] == o
                assert len(run_chain(adj, plan["chain"])) == want, (name, o, fl)


def test_chain_listing_equals_oracle_matches():
    g = oracle.relabel_by_degree(inputs.gnp(20, 1, 3, 5))[0]
    adj = _adj_sets(g)
    for name in ["c4", "house", "tailed_diamond_a", "diamond"]:
        k, e = Q[name]
        po = oracle.symmetry_breaking_order(k, e)
        o = oracle.connected_order(k, e)
        plan = huge.plan_offline(k, e, order=o, po=po)
        got = to_query_order(run_chain(adj, plan["chain"]), plan["chain"]["order"])
        want = oracle.list_matches(g, k, e, po)
        assert np.array_equal(_sorted_rows(got), _sorted_rows(want)), name


def test_automatic_partial_order_breaks_every_symmetry():
    """The library's own partial order (npo = -1): count x |Aut(Q)| = the count without any."""
    g = oracle.relabel_by_degree(inputs.gnp(22, 1, 3, 8))[0]
    adj = _adj_sets(g)
    for s in range(16):
        k, e = inputs.random_query(3 + s % 3, 900 + s)
        plan = huge.plan_offline(k, e, order=oracle.connected_order(k, e))
        aut = len(oracle.automorphisms(k, e))
        assert len(run_chain(adj, plan["chain"])) * aut == oracle.count(g, k, e, []), (k, e)


def _closure(k, po):
    lt = np.zeros((k, k), dtype=bool)
    for a, b in po:
        lt[a, b] = True
    for m in range(k):
        lt |= lt[:, [m]] & lt[[m], :]
    return lt


@pytest.mark.parametrize("name", ["c4", "path4", "house", "c5", "path5", "c6", "tailed_diamond_a"])
def test_push_join_plans_match_oracle(name):
    """Forced PUSH-JOIN plans under several cardinality tables (so several splits and build
    sides): the joined rows are exactly the oracle's matches."""
    g = oracle.relabel_by_degree(inputs.gnp(18, 1, 3, 40))[0]
    adj = _adj_sets(g)
    k, e = Q[name]
    po = oracle.symmetry_breaking_order(k, e)
    want = _sorted_rows(oracle.list_matches(g, k, e, po))
    rng = np.random.default_rng(3)
    splits = set()
    for t in range(6):
        card = rng.uniform(1.0, 1e6, 1 << k)
        plan = huge.plan_offline(k, e, po=po, flags=huge.PLAN_FORCE_JOIN, card=card, edges_g=100.0)
        assert plan["op"] == "PUSH-JOIN"
        splits.add((tuple(plan["left_vertices"]), tuple(plan["right_vertices"])))
        got = _sorted_rows(run_join(adj, plan))
        assert np.array_equal(got, want), (name, plan["left_vertices"], plan["right_vertices"])
    assert len(splits) >= 2 or name in ("c4",), splits


DOWN_PENALTY = 0.25  # the optimiser's charge for an extension bounded only from above
UPPER_PENALTY = 0.05  # ... and for one bounded from both sides


def _connected(es, m):
    vs = [v for v in range(8) if m >> v & 1]
    seen, todo = {vs[0]}, [vs[0]]
    while todo:
        u = todo.pop()
        for v in vs:
            if v not in seen and frozenset((u, v)) in es:
                seen.add(v)
                todo.append(v)
    return len(seen) == len(vs)


def _order_cost(order, card, lt, edges_g):
    """Cost of the EXTEND chain of one matching order in Alg. 1's model: the first edge's
    cardinality, then per extension |R(prefix)| + |E_G| (+ the tie-breaking bound penalties)."""
    m = (1 << order[0]) | (1 << order[1])
    cost = card[m]
    for v in order[2:]:
        lo = any(lt[u, v] for u in range(len(lt)) if m >> u & 1)
        hi = any(lt[v, u] for u in range(len(lt)) if m >> u & 1)
        m |= 1 << v
        cost += card[m] + edges_g + ((UPPER_PENALTY if lo else DOWN_PENALTY) * card[m] if hi else 0.0)
    return cost


@functools.lru_cache(maxsize=None)
def _best_chain_cost_cached(es, mask, card_t, lt_t, edges_g):
    return _best_chain_cost(es, mask, np.asarray(card_t), np.asarray(lt_t), edges_g)


def _best_chain_cost(es, mask, card, lt, edges_g):
    vs = [v for v in range(8) if mask >> v & 1]
    best = None
    for o in itertools.permutations(vs):
        ok = all(any(frozenset((o[j], o[t])) in es for t in range(j)) for j in range(1, len(o)))
        if ok:
            c = _order_cost(list(o), card, lt, edges_g)
            best = c if best is None else min(best, c)
    return best


@pytest.mark.parametrize("seed", range(12))  # seed 9: a PUSH-JOIN at the top is cheapest
def test_optimiser_equals_exhaustive_search(seed):
    """Alg. 1's dynamic programme over sub-queries finds the cheapest plan that trying every
    matching order, and every PUSH-JOIN split of the whole query, finds."""
    rng = np.random.default_rng(100 + seed)
    k = 4 + seed % 3
    _, e = inputs.random_query(k, 7000 + seed, 1, 3)
    es = {frozenset(x) for x in map(tuple, e)}
    card = np.exp(rng.uniform(0, 40, 1 << k))
    edges_g = float(rng.uniform(10, 1e4))
    plan_x = huge.plan_offline(k, e, flags=huge.PLAN_EXTEND_ONLY, card=card, edges_g=edges_g)
    lt = _closure(k, [tuple(p) for p in plan_x["po"]])
    full = (1 << k) - 1
    best_ext = _best_chain_cost(es, full, card, lt, edges_g)
    assert plan_x["op"] == "EXTEND-CHAIN"
    assert plan_x["est_cost"] == pytest.approx(best_ext, rel=1e-9)
    assert _order_cost(plan_x["chain"]["order"], card, lt, edges_g) == pytest.approx(best_ext, rel=1e-9)
    # PUSH-JOIN at the top: key K = L & R an independent set of <= 4 vertices, no edge between
    # the two sides' non-key vertices
    best_join = None
    for L in range(1, full):
        for R in range(1, full):
            K = L & R
            if (L | R) != full or not K or K == L or K == R or bin(K).count("1") > 4:
                continue
            if bin(L).count("1") < 2 or bin(R).count("1") < 2 or not _connected(es, L) or not _connected(es, R):
                continue
            if any(K >> a & 1 and K >> b & 1 for a, b in map(tuple, e)):
                continue
            if any((L & ~K) >> a & 1 and (R & ~K) >> b & 1 or (L & ~K) >> b & 1 and (R & ~K) >> a & 1
                   for a, b in map(tuple, e)):
                continue
            key = (frozenset(es), tuple(card), tuple(map(tuple, lt)), edges_g)
            c = (_best_chain_cost_cached(key[0], L, *key[1:]) + _best_chain_cost_cached(key[0], R, *key[1:])
                 + card[full] + card[L] + card[R])
            best_join = c if best_join is None else min(best_join, c)
    plan = huge.plan_offline(k, e, card=card, edges_g=edges_g)
    best = best_ext if best_join is None else min(best_ext, best_join)
    assert plan["est_cost"] == pytest.approx(best, rel=1e-9)
    assert plan["op"] == ("PUSH-JOIN" if best_join is not None and best_join < best_ext else "EXTEND-CHAIN")


def test_offline_rejects_bad_input():
    k, e = Q["c4"]
    with pytest.raises(huge.HugeError) as ei:
        huge.plan_offline(k, e)  # neither an order nor cardinalities
    assert ei.value.code == huge.EINVAL
    with pytest.raises(huge.HugeError):
        huge.plan_offline(k, e, order=[0, 2, 1, 3])  # prefix {0, 2} is not connected
    with pytest.raises(huge.HugeError):
        huge.plan_offline(k, e, order=[0, 1, 2, 3], po=[(0, 1), (1, 0)])  # not a DAG
    with pytest.raises(huge.HugeError) as ei:
        huge.plan_offline(k, e, order=[0, 1, 2, 3], po=[(0, 9)])  # vertex 9 is not in the query
    assert ei.value.code == huge.EINVAL
    with pytest.raises(huge.HugeError):
        huge.plan_offline(3, [(0, 1)], order=[0, 1, 2])  # disconnected query
    with pytest.raises(huge.HugeError) as ei:
        huge.plan_offline(4, Q["k4"][1], card=np.ones(16), flags=huge.PLAN_FORCE_JOIN)  # no valid split
    assert ei.value.code == huge.EINVAL


def test_arbitrary_partial_orders_and_orders_match_oracle():
    """Any acyclic partial order a caller gives (not only a symmetry-breaking one), including
    pairs implied only transitively, with any connected matching order."""
    g = oracle.relabel_by_degree(inputs.gnp(16, 1, 3, 12))[0]
    adj = _adj_sets(g)
    rng = np.random.default_rng(12)
    for s in range(40):
        k = 3 + s % 3
        _, e = inputs.random_query(k, 3000 + s)
        rank = rng.permutation(k)  # pairs a < b only when rank[a] < rank[b]: acyclic
        pairs = [(a, b) for a in range(k) for b in range(k) if rank[a] < rank[b] and rng.random() < 0.35]
        orders = list(connected_orders(k, e))
        o = orders[int(rng.integers(len(orders)))]
        plan = huge.plan_offline(k, e, order=o, po=pairs, flags=huge.PLAN_TREE_VERIFY if s % 2 else 0)
        assert len(run_chain(adj, plan["chain"])) == oracle.count(g, k, e, pairs), (k, e, pairs, o)


def test_connected_orders_of_the_regret_evaluation():
    """The regret evaluation scores every matching order with connected prefixes, the same list
    brute force over all permutations gives (24 for K4; 16 for C4: any start, then either
    neighbour, and so on)."""
    import itertools

    from paper_2103_14294_b300 import learned

    for name in ("k4", "c4", "house", "path4", "star4"):
        k, e = inputs.QUERIES[name]
        es = {frozenset(x) for x in e}
        want = [list(o) for o in itertools.permutations(range(k))
                if all(any(frozenset((o[j], o[t])) in es for t in range(j)) for j in range(1, k))]
        assert learned.connected_orders(k, e) == want
    assert len(learned.connected_orders(4, inputs.QUERIES["k4"][1])) == 24
    assert len(learned.connected_orders(4, inputs.QUERIES["c4"][1])) == 16


# ---- directed plans (HUGE_PLAN_DIRECTED): the same interpreter with out- and in-lists ----

DIRECTED_QUERIES = {
    "cycle3": (3, [(0, 1), (1, 2), (2, 0)]),
    "transitive3": (3, [(0, 1), (1, 2), (0, 2)]),
    "in_star3": (4, [(1, 0), (2, 0), (3, 0)]),
    "cycle4": (4, [(0, 1), (1, 2), (2, 3), (3, 0)]),
    "bifan": (4, [(0, 2), (0, 3), (1, 2), (1, 3)]),
    "two_cycle_tail": (3, [(0, 1), (1, 0), (1, 2)]),
    "feedback4": (4, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 1)]),
}


def run_chain_directed(out_adj, in_adj, chain):
    """run_chain for a directed plan: list j of an EXTEND is the in-list of its position's vertex
    when dirs[j] is 1, else its out-list; a VERIFY pair (a, b) needs the arc f[a] -> f[b], or
    f[b] -> f[a] when its bit is 1."""
    rows = [(r,) for r in range(len(out_adj))]
    for st in chain["steps"]:
        dirs = st.get("dirs", [0] * len(st["ext"]))
        lists = lambda f: [(in_adj if d else out_adj)[f[p]] for p, d in zip(st["ext"], dirs)]
        out = []
        if st["op"] == "EXTEND":
            for f in rows:
                for u in set.intersection(*lists(f)):
                    if all(u > f[p] for p in st["lo"]) and all(u < f[p] for p in st["hi"]) and \
                            all(u != f[p] for p in st["inj"]):
                        out.append(f + (u,))
        else:
            out = [f for f in rows
                   if all(f[b] in (in_adj if d else out_adj)[f[a]] for a, b, d in zip(st["ext"], st["with"], dirs))]
        rows = out
    return rows


@pytest.mark.parametrize("seed", [1, 2])
def test_directed_chain_plans_of_every_order_match_oracle(seed):
    g = inputs.gnp_directed(16, 1, 4, 50 + seed)
    out_adj = _adj_sets(g)
    in_adj = _adj_sets(oracle.reverse_csr(g))
    for name, (k, a) in DIRECTED_QUERIES.items():
        po = oracle.symmetry_breaking_order(k, a, directed=True)
        want = oracle.count_directed(g, k, a, po)
        for o in connected_orders(k, a):
            for fl in (huge.PLAN_PLAIN, huge.PLAN_TREE_VERIFY):
                plan = huge.plan_offline(k, a, order=o, flags=fl | huge.PLAN_DIRECTED)
                assert len(run_chain_directed(out_adj, in_adj, plan["chain"])) == want, (name, o, fl)


def test_directed_automatic_order_and_reversed_arcs():
    """The library's automatic partial order of a directed query breaks exactly its
    arc-preserving automorphisms; a query with every arc reversed is a different query."""
    g = inputs.gnp_directed(14, 1, 3, 9)
    out_adj, in_adj = _adj_sets(g), _adj_sets(oracle.reverse_csr(g))
    for name, (k, a) in DIRECTED_QUERIES.items():
        aut = len(oracle.automorphisms(k, a, directed=True))
        plan = huge.plan_offline(k, a, order=oracle.connected_order(k, a), flags=huge.PLAN_DIRECTED)
        assert len(run_chain_directed(out_adj, in_adj, plan["chain"])) * aut == oracle.count_directed(g, k, a)
    # in the out-star every arc leaves the centre; the in-star's arcs enter it: different counts
    k, a = DIRECTED_QUERIES["in_star3"]
    rev = [(y, x) for x, y in a]
    p1 = huge.plan_offline(k, a, order=[0, 1, 2, 3], po=[], flags=huge.PLAN_DIRECTED)
    p2 = huge.plan_offline(k, rev, order=[0, 1, 2, 3], po=[], flags=huge.PLAN_DIRECTED)
    assert len(run_chain_directed(out_adj, in_adj, p1["chain"])) == oracle.count_directed(g, k, a)
    assert len(run_chain_directed(out_adj, in_adj, p2["chain"])) == oracle.count_directed(g, k, rev)
    with pytest.raises(huge.HugeError):  # K5 with both arcs per edge: 8 lists at a vertex
        kk, e = Q["k5"]
        huge.plan_offline(kk, e + [(y, x) for x, y in e], order=[0, 1, 2, 3, 4], flags=huge.PLAN_DIRECTED)


def run_chain_labeled(adj, chain):
    """run_chain for a labelled plan on a graph whose ids are grouped by label: roots lie in the
    chain's "root" range and an EXTEND's new vertex in its "ids" range (both half-open)."""
    lo, hi = chain.get("root", [0, len(adj)])
    rows = [(r,) for r in range(len(adj)) if lo <= r < hi]
    for st in chain["steps"]:
        out = []
        if st["op"] == "EXTEND":
            ilo, ihi = st.get("ids", [0, len(adj)])
            for f in rows:
                for u in set.intersection(*[adj[f[p]] for p in st["ext"]]):
                    if ilo <= u < ihi and all(u > f[p] for p in st["lo"]) and \
                            all(u < f[p] for p in st["hi"]) and all(u != f[p] for p in st["inj"]):
                        out.append(f + (u,))
        else:
            out = [f for f in rows if all(f[b] in adj[f[a]] for a, b in zip(st["ext"], st["with"]))]
        rows = out
    return rows


@pytest.mark.parametrize("seed", [1, 2])
def test_labelled_chain_plans_of_every_order_match_oracle(seed):
    """Label bounds compiled for every matching order (Sec. 2: a labelled query vertex only
    admits data vertices of its label) give the oracle's labelled count, which checks the label
    of each assignment directly. Ranges of unequal sizes, a wildcard and a label no vertex
    carries are included."""
    g = inputs.gnp(30, 1, 4, 70 + seed)
    lstart = [0, 7, 19, 30]  # label L owns ids [lstart[L], lstart[L + 1])
    dl = np.repeat(np.arange(3, dtype=np.uint32), np.diff(lstart))
    adj = _adj_sets(g)
    rng = np.random.default_rng(seed)
    any_l = oracle.ANY_LABEL
    for name in ["triangle", "c4", "diamond", "house", "tailed_triangle", "path4"]:
        k, e = Q[name]
        for trial in range(3):
            ql = [int(x) for x in rng.integers(0, 3, k)]
            if trial == 1:
                ql[int(rng.integers(k))] = any_l
            po = oracle.symmetry_breaking_order(k, e, ql)
            want = oracle.count(g, k, e, po, dlabels=dl, qlabels=ql)
            for o in connected_orders(k, e):
                for fl in (huge.PLAN_PLAIN, huge.PLAN_TREE_VERIFY):
                    plan = huge.plan_offline(k, e, order=o, flags=fl, labels=ql, lstart=lstart)
                    assert len(run_chain_labeled(adj, plan["chain"])) == want, (name, ql, o, fl)
    # a label beyond the graph's: empty range, no match
    k, e = Q["triangle"]
    plan = huge.plan_offline(k, e, order=[0, 1, 2], labels=[0, 5, 1], lstart=lstart)
    assert len(run_chain_labeled(adj, plan["chain"])) == 0
    with pytest.raises(huge.HugeError):  # ranges that decrease
        huge.plan_offline(k, e, order=[0, 1, 2], labels=[0, 1, 1], lstart=[0, 9, 4, 30])


def test_labelled_automatic_order_breaks_only_label_preserving_symmetry():
    """A triangle with two equal labels keeps one symmetry of 6; with three distinct labels none:
    the automatic partial order, run by the interpreter, times |Aut| gives the count with no
    order at all."""
    g = inputs.gnp(30, 1, 3, 91)
    lstart = [0, 10, 20, 30]
    dl = np.repeat(np.arange(3, dtype=np.uint32), np.diff(lstart))
    adj = _adj_sets(g)
    k, e = Q["triangle"]
    for ql in ([0, 0, 1], [0, 1, 2], [2, 2, 2]):
        aut = len(oracle.automorphisms(k, e, ql))
        plan = huge.plan_offline(k, e, order=[0, 1, 2], labels=ql, lstart=lstart)
        got = len(run_chain_labeled(adj, plan["chain"]))
        assert got * aut == oracle.count(g, k, e, [], dlabels=dl, qlabels=ql), ql


def _exact_cards(g, k, e, po):
    """|R(q')| of every connected sub-query q' (the query induced on a vertex mask, with the
    partial order restricted to it), counted by the oracle: the exact values Alg. 1's
    cardinality estimator stands in for."""
    es = {frozenset(x) for x in map(tuple, e)}
    lt = _closure(k, po)
    card = np.zeros(1 << k)
    for m in range(1, 1 << k):
        vs = [v for v in range(k) if m >> v & 1]
        if len(vs) < 2 or not _connected(es, m):
            continue
        idx = {v: i for i, v in enumerate(vs)}
        se = [(idx[a], idx[b]) for a, b in map(tuple, e) if a in idx and b in idx]
        spo = [(idx[a], idx[b]) for a in vs for b in vs if lt[a, b]]
        card[m] = float(oracle.count(g, len(vs), se, spo))
    return card


@pytest.mark.parametrize("graph", ["rmat", "er"])
def test_alg1_example_plans_of_the_4clique_and_the_5path(graph):
    """Alg. 1's worked example (Sec. 3.3, the example plans of the 4-clique and the 5-path):
    with the true sub-query cardinalities of a data graph, the optimal plan of the 4-clique is
    a chain of pulling extensions, each a complete star join of every bound vertex; the optimal
    plan of the 5-path is hybrid, a pushing hash join (PUSH-JOIN) on top of pulling extensions,
    and its joined rows are the oracle's matches."""
    g0 = inputs.rmat(10, 8, 3) if graph == "rmat" else inputs.er(200, 800, 4)
    g = oracle.relabel_by_degree(g0)[0]
    edges_g = g.nnz / 2
    k, e = Q["k4"]
    po = oracle.symmetry_breaking_order(k, e)
    plan = huge.plan_offline(k, e, po=po, card=_exact_cards(g, k, e, po), edges_g=edges_g)
    assert plan["op"] == "EXTEND-CHAIN"
    assert [sorted(s["ext"]) for s in plan["chain"]["steps"]] == [[0], [0, 1], [0, 1, 2]]
    k, e = Q["path5"]
    po = oracle.symmetry_breaking_order(k, e)
    plan = huge.plan_offline(k, e, po=po, card=_exact_cards(g, k, e, po), edges_g=edges_g)
    assert plan["op"] == "PUSH-JOIN"
    assert all(s["op"] == "EXTEND" for side in ("left", "right") for s in plan[side]["steps"])
    assert len(plan["join_spec"]["lkey"]) == 1  # the two sides share one vertex
    if graph == "er":  # small enough to list every match
        adj = _adj_sets(g)
        want = _sorted_rows(oracle.list_matches(g, k, e, po))
        assert np.array_equal(_sorted_rows(run_join(adj, plan)), want)


def _clique(k):
    return [(a, b) for a in range(k) for b in range(a + 1, k)]


def _cycle(k):
    return [(i, (i + 1) % k) for i in range(k)]


@pytest.mark.parametrize("name,k,edges,graph", [
    ("k7", 7, _clique(7), (13, 3, 4, 5)),
    ("k8", 8, _clique(8), (12, 9, 10, 1)),
    ("c8", 8, _cycle(8), (16, 1, 4, 7)),
    ("wheel8", 8, _cycle(7) + [(7, i) for i in range(7)], (14, 2, 3, 8)),
])
def test_largest_queries_compile_to_exact_chains(name, k, edges, graph):
    """Queries of the largest supported size (8 vertices, up to 7 lists in one EXTEND): sampled
    matching orders, plain and verify-only, give the oracle's count through the interpreter."""
    g = oracle.relabel_by_degree(inputs.gnp(*graph))[0]
    adj = _adj_sets(g)
    po = oracle.symmetry_breaking_order(k, edges)
    want = oracle.count(g, k, edges, po)
    assert want > 0
    orders = list(connected_orders(k, edges))
    rng = np.random.default_rng(k)
    for i in rng.choice(len(orders), 4, replace=False):
        for fl in (huge.PLAN_PLAIN, huge.PLAN_TREE_VERIFY):
            plan = huge.plan_offline(k, edges, order=orders[i], flags=fl)
            assert len(run_chain(adj, plan["chain"])) == want, (name, orders[i], fl)
    with pytest.raises(huge.HugeError):  # one vertex more than the limit
        huge.plan_offline(9, _cycle(9), order=list(range(9)))


def test_labelled_directed_chain_plans_of_every_order_match_oracle():
    """Labels and arcs compiled together: each EXTEND list is an out-list or in-list by its arc,
    and the new vertex lies in its label's id range; every order, plain and verify-only."""
    g = inputs.gnp_directed(21, 1, 3, 64)
    lstart = [0, 6, 13, 21]
    dl = np.repeat(np.arange(3, dtype=np.uint32), np.diff(lstart))
    out_adj, in_adj = _adj_sets(g), _adj_sets(oracle.reverse_csr(g))
    rng = np.random.default_rng(4)
    for name, (k, a) in DIRECTED_QUERIES.items():
        ql = [int(x) for x in rng.integers(0, 3, k)]
        po = oracle.symmetry_breaking_order(k, a, ql, directed=True)
        want = oracle.count_directed(g, k, a, po, dlabels=dl, qlabels=ql)
        for o in connected_orders(k, a):
            for fl in (huge.PLAN_PLAIN, huge.PLAN_TREE_VERIFY):
                plan = huge.plan_offline(k, a, order=o, flags=fl | huge.PLAN_DIRECTED, labels=ql, lstart=lstart)
                chain = plan["chain"]
                lo, hi = chain.get("root", [0, g.n])
                rows = [(r,) for r in range(g.n) if lo <= r < hi]
                for st in chain["steps"]:
                    dirs = st.get("dirs", [0] * len(st["ext"]))
                    lists = lambda f: [(in_adj if d else out_adj)[f[p]] for p, d in zip(st["ext"], dirs)]
                    if st["op"] == "EXTEND":
                        ilo, ihi = st.get("ids", [0, g.n])
                        rows = [f + (u,) for f in rows for u in set.intersection(*lists(f))
                                if ilo <= u < ihi and all(u > f[p] for p in st["lo"]) and
                                all(u < f[p] for p in st["hi"]) and all(u != f[p] for p in st["inj"])]
                    else:
                        rows = [f for f in rows if all(f[b] in (in_adj if d else out_adj)[f[x]]
                                                       for x, b, d in zip(st["ext"], st["with"], dirs))]
                assert len(rows) == want, (name, ql, o, fl)
