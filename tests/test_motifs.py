"""Motif counting (graph pattern mining, Sec. 6) on the CPU: the oracle's census pinned by
closed forms, the pattern catalogue and containment numbers pinned by counting facts about
labelled graphs, and the library's non-induced -> induced conversion checked against the
oracle's census, using the oracle's non-induced counts as input."""
from math import comb

import numpy as np
import pytest

import inputs
import oracle
from paper_2103_14294_b300 import motifs


def graph_of(n, edges):
    nbr = [[] for _ in range(n)]
    for a, b in edges:
        nbr[a].append(b)
        nbr[b].append(a)
    off = np.zeros(n + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(x) for x in nbr])
    adj = np.asarray([v for x in nbr for v in sorted(x)], dtype=np.uint32)
    return inputs.Graph(off, adj, "test")


def key(k, edges):
    return oracle.motif_key(k, edges)


PATH = {k: [(i, i + 1) for i in range(k - 1)] for k in (3, 4, 5)}
STAR = {k: [(0, i) for i in range(1, k)] for k in (3, 4, 5)}
CLIQUE = {k: [(i, j) for i in range(k) for j in range(i + 1, k)] for k in (3, 4, 5)}


@pytest.mark.parametrize("k", [3, 4, 5])
def test_oracle_census_closed_forms(k):
    n = 9
    assert oracle.motif_census(inputs.complete(n), k) == {key(k, CLIQUE[k]): comb(n, k)}
    cycle = graph_of(n, [(i, (i + 1) % n) for i in range(n)])
    assert oracle.motif_census(cycle, k) == {key(k, PATH[k]): n}
    star = graph_of(n, [(0, i) for i in range(1, n)])
    assert oracle.motif_census(star, k) == {key(k, STAR[k]): comb(n - 1, k - 1)}


def test_oracle_census_complete_bipartite():
    a, b = 4, 5
    g = inputs.complete_bipartite(a, b)
    assert oracle.motif_census(g, 3) == {key(3, PATH[3]): a * comb(b, 2) + b * comb(a, 2)}
    c4 = [(0, 1), (1, 2), (2, 3), (3, 0)]
    assert oracle.motif_census(g, 4) == {key(4, c4): comb(a, 2) * comb(b, 2),
                                         key(4, STAR[4]): a * comb(b, 3) + b * comb(a, 3)}


def test_pattern_catalogue_and_containment():
    # connected unlabelled graphs on 3, 4, 5 vertices: 2, 6, 21
    assert [len(motifs.patterns(k)) for k in (3, 4, 5)] == [2, 6, 21]
    for k, connected_labelled in ((3, 4), (4, 38), (5, 728)):
        c = motifs.containment(k)
        clique = motifs.pattern_index(k, CLIQUE[k])
        # every connected spanning subgraph of K_k is a copy of exactly one pattern
        assert sum(c[i][clique] for i in range(len(c))) == connected_labelled
        # spanning trees of K_k: k^(k-2) (Cayley)
        trees = [i for i, p in enumerate(motifs.patterns(k)) if len(p) == k - 1]
        assert sum(c[i][clique] for i in trees) == k ** (k - 2)
        # Hamiltonian paths of K_k: k!/2
        assert c[motifs.pattern_index(k, PATH[k])][clique] == {3: 3, 4: 12, 5: 60}[k]
        for i in range(len(c)):
            assert c[i][i] == 1 and all(c[i][j] == 0 for j in range(i))


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("k", [3, 4, 5])
def test_induced_from_noninduced_matches_oracle_census(k, seed):
    g = inputs.gnp(13, 1, 3, 60 + seed)
    nonind = [oracle.count(g, k, list(p), oracle.symmetry_breaking_order(k, list(p))) for p in motifs.patterns(k)]
    ind = motifs.induced_from_noninduced(k, nonind)
    want = oracle.motif_census(g, k)
    got = {key(k, p): c for p, c in zip(motifs.patterns(k), ind) if c}
    assert got == want


def test_inconsistent_counts_rejected():
    with pytest.raises(ValueError):
        motifs.induced_from_noninduced(3, [0, 5])  # five triangles but no wedges


@pytest.mark.parametrize("k", [3, 4, 5])
def test_census_plans_interpreted_on_host_match_oracle(k):
    """The plans the census launches (each pattern's connected order and automatic partial
    order), compiled by the host planner and run by a plain interpreter, give the census."""
    from paper_2103_14294_b300 import huge
    from test_plan_host import _adj_sets, run_chain

    g = oracle.relabel_by_degree(inputs.gnp(14, 1, 3, 17))[0]
    adj = _adj_sets(g)
    nonind = []
    for p in motifs.patterns(k):
        plan = huge.plan_offline(k, list(p), order=motifs._order(k, p))
        nonind.append(len(run_chain(adj, plan["chain"])))
    got = {key(k, p): c for p, c in zip(motifs.patterns(k), motifs.induced_from_noninduced(k, nonind)) if c}
    assert got == oracle.motif_census(g, k)
