"""Motif counting on top of the enumerator (Sec. 6, graph pattern mining).

A motif census of size k counts, for every connected pattern H on k vertices, the k-vertex sets
of the data graph whose induced subgraph is isomorphic to H. HUGE serves pattern mining by
running subgraph enumeration over the small patterns; here all patterns of one size go to the
GPU as one batched persistent launch, each pattern with its symmetry-breaking partial order, so
every count is the number of (non-induced) subgraphs isomorphic to H.

Non-induced and induced counts are related through the patterns that contain one another on the
same k vertices: nonind(H) = sum over patterns H' of c(H, H') * ind(H'), with c(H, H') the number
of spanning subgraphs of H' isomorphic to H (non-zero only when H' has at least H's edges). The
system is triangular in the edge count and is solved exactly in integers, densest pattern first.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

from . import huge

MAX_K = 5


def _relabel(edges, perm):
    return tuple(sorted(tuple(sorted((perm[a], perm[b]))) for a, b in edges))


def _connected(k, edges):
    adj = {v: set() for v in range(k)}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    seen, todo = {0}, [0]
    while todo:
        for w in adj[todo.pop()] - seen:
            seen.add(w)
            todo.append(w)
    return len(seen) == k


def canonical(k, edges):
    """The lexicographically smallest sorted edge tuple over all relabellings (k <= 5)."""
    return min(_relabel(edges, p) for p in itertools.permutations(range(k)))


@lru_cache(maxsize=None)
def patterns(k: int):
    """Every connected graph on k vertices up to isomorphism (canonical edge tuples), ordered
    by edge count, then lexicographically: 2, 6 and 21 patterns for k = 3, 4, 5."""
    if not 2 <= k <= MAX_K:
        raise ValueError(f"motif size must be 2..{MAX_K}")
    pairs = list(itertools.combinations(range(k), 2))
    found = set()
    for bits in range(1, 1 << len(pairs)):
        es = [pairs[i] for i in range(len(pairs)) if bits >> i & 1]
        if len(es) >= k - 1 and _connected(k, es):
            found.add(canonical(k, es))
    return tuple(sorted(found, key=lambda e: (len(e), e)))


def _maps_into(k, eh, eg):
    """Bijections of the k vertices sending every edge of eh to an edge of eg."""
    g = {frozenset(e) for e in eg}
    return sum(all(frozenset((p[a], p[b])) in g for a, b in eh) for p in itertools.permutations(range(k)))


@lru_cache(maxsize=None)
def containment(k: int):
    """c[i][j] = the number of spanning subgraphs of pattern j isomorphic to pattern i."""
    ps = patterns(k)
    aut = [_maps_into(k, p, p) for p in ps]
    return tuple(tuple(_maps_into(k, ps[i], ps[j]) // aut[i] for j in range(len(ps))) for i in range(len(ps)))


def induced_from_noninduced(k: int, noninduced):
    """Induced counts from non-induced ones (both indexed like patterns(k)), in exact integers."""
    c = containment(k)
    n = len(c)
    ind = [0] * n
    for i in reversed(range(n)):
        rest = int(noninduced[i]) - sum(c[i][j] * ind[j] for j in range(i + 1, n))
        if rest < 0:
            raise ValueError("non-induced counts are inconsistent (a count is too small)")
        ind[i] = rest  # c[i][i] = 1
    return ind


def _order(k, edges):
    """A connected matching order: breadth first from vertex 0."""
    adj = {v: set() for v in range(k)}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    order, seen = [0], {0}
    for v in order:
        for w in sorted(adj[v] - seen):
            seen.add(w)
            order.append(w)
    return order


def census(graph: huge.Graph, k: int, mem_bound: int = 1 << 30, stream=None):
    """Motif census of size k on a loaded graph: a list of (pattern edges, non-induced count,
    induced count), one per connected pattern, from one batched launch."""
    ps = patterns(k)
    plans = [huge.Plan(graph, k, list(p), order=_order(k, p)) for p in ps]
    try:
        nonind = huge.enumerate_batch(plans, mem_bound=mem_bound, stream=stream)
    finally:
        for p in plans:
            p.free()
    ind = induced_from_noninduced(k, [int(x) for x in nonind])
    return [(list(p), int(a), int(b)) for p, a, b in zip(ps, nonind, ind)]


def pattern_index(k: int, edges) -> int:
    """Position of the pattern isomorphic to `edges` in patterns(k)."""
    return patterns(k).index(canonical(k, edges))
