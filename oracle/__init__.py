"""CPU oracle for subgraph enumeration — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of ``bench.py`` may
import this package. The library under ``paper_2103_14294_b300`` never does, and the two share
no code: the oracle has its own relabelling, its own automorphism search and its own
symmetry-breaking partial order, written from the paper's definitions.

Functions and what they follow:

* ``count`` / ``count_roots`` / ``list_matches`` — the definition of a match (Sec. 2,
  "Subgraph Enumeration"): an injective map sending query edges to data edges, restricted by
  the partial order of symmetry breaking (Sec. 2). Plain backtracking in C (``oracle.c``).
* ``brute`` — the same definition by trying every tuple of distinct vertices (tiny graphs).
* ``relabel_by_degree`` — the data total order of Sec. 2: smaller degree gets the smaller id,
  ties broken by the original id.
* ``automorphisms`` — all permutations of the query's vertices that preserve its edge set,
  by trying every permutation (queries of at most 8 vertices).
* ``symmetry_breaking_order`` — the partial order of symmetry breaking (the paper cites
  Grochow & Kellis for it): pick the smallest vertex with a non-trivial orbit under the
  remaining automorphism group, require it to be below every other vertex of its orbit,
  restrict the group to its stabiliser, repeat until the group is trivial.
* ``motif_census`` / ``motif_key`` — the induced motif census by its definition (graph
  pattern mining, Sec. 6): every k-vertex subset whose induced subgraph is connected, counted
  per isomorphism class (classes told apart by the smallest adjacency bitmask over all
  relabellings). Tiny graphs only.
* ``prefix_counts`` — |R(q'_i)| for every prefix q'_i of a matching order (the partial
  results an EXTEND chain produces, Sec. 3.1 Eq. 2 and Sec. 4.2), each the count of the
  induced prefix sub-query with the partial-order pairs inside the prefix.

* ``count(..., dlabels, qlabels)`` / ``brute_labeled`` — labelled matches (Sec. 2 notes the
  method carries over to labelled graphs): additionally label(f(v)) = qlabels[v], with
  ANY_LABEL matching every label; symmetry breaking then uses the label-preserving
  automorphisms (``automorphisms(k, edges, labels)``).
* ``count_directed`` / ``brute_directed`` — directed queries on directed graphs: every query
  arc a -> b must map to a data arc f(a) -> f(b); the backtracker scans a parent's out-list or
  in-list (``reverse_csr``) by the arc's direction; symmetry breaking uses the arc-preserving
  automorphisms (arc- and label-preserving with labels, which both functions also take).
* ``walk_traces`` / ``triangle_count_trace`` / ``c4_count_trace`` — whole-graph counts from
  closed walks of the adjacency matrix, with no enumeration: tr(A^3) = 6 #K3 and
  tr(A^4) = 8 #C4 + 2m + 4 sum_v C(d(v), 2) (textbook identities; the 4-cycle and the triangle
  are the square and the clique of Sec. 7's queries).
* ``clique_count`` — number of k-cliques by the textbook degree-orientation method (Chiba and
  Nishizeki): each clique counted once from its smallest vertex in (degree, id) order. It
  shares nothing with the backtracker and serves as a second, independent count of K4 / K5.

* ``oracle.scheduler`` — Alg. 5 (the DFS/BFS-adaptive scheduler) as a host model over
  bounded batch queues, with SCAN / EXTEND / SINK operators built from the definition of a
  match; its own module docstring states the rules it follows.

Pins (checked in ``tests/test_oracle.py`` against facts that do not come from this code):
closed forms on complete and complete bipartite graphs (also two-coloured and directed ones),
brute force on tiny graphs (unlabelled, labelled, directed, both), the automorphism invariant,
the labelling partition identity, trace identities of the adjacency matrix, prefix counts
level by level against brute force, and for the scheduler model the running example of
Sec. 5.2 slot by slot plus the backtracker's counts. The stored golden counts that take
seconds are re-derived there too.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_count.argtypes = [ctypes.c_uint32, P, P, ctypes.c_int, P, P, ctypes.c_int, P,
                                         ctypes.c_uint32, ctypes.c_uint32, P, ctypes.c_int]
            lib.oracle_count.restype = ctypes.c_int64
            lib.oracle_count_roots.argtypes = [ctypes.c_uint32, P, P, ctypes.c_int, P, P, ctypes.c_int,
                                               P, P, ctypes.c_uint64, P, ctypes.c_int]
            lib.oracle_count_roots.restype = ctypes.c_int64
            lib.oracle_list.argtypes = [ctypes.c_uint32, P, P, ctypes.c_int, P, P, ctypes.c_int, P, P,
                                        ctypes.c_uint64]
            lib.oracle_list.restype = ctypes.c_int64
            lib.oracle_brute.argtypes = [ctypes.c_uint32, P, P, ctypes.c_int, P, ctypes.c_int, P]
            lib.oracle_brute.restype = ctypes.c_int64
            lib.oracle_count_labeled.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_int, P, P, P, ctypes.c_int, P,
                                                 ctypes.c_uint32, ctypes.c_uint32, P, ctypes.c_int]
            lib.oracle_count_labeled.restype = ctypes.c_int64
            lib.oracle_brute_labeled.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_int, P, P, ctypes.c_int, P]
            lib.oracle_brute_labeled.restype = ctypes.c_int64
            lib.oracle_count_directed.argtypes = [ctypes.c_uint32, P, P, P, P, P, ctypes.c_int, P, P, P,
                                                  ctypes.c_int, P, ctypes.c_uint32, ctypes.c_uint32, P, ctypes.c_int]
            lib.oracle_count_directed.restype = ctypes.c_int64
            lib.oracle_brute_directed.argtypes = [ctypes.c_uint32, P, P, P, ctypes.c_int, P, P, ctypes.c_int, P]
            lib.oracle_brute_directed.restype = ctypes.c_int64
            lib.oracle_walk_traces.argtypes = [ctypes.c_uint32, P, P, ctypes.c_int, P]
            lib.oracle_walk_traces.restype = ctypes.c_int
            lib.oracle_clique_count.argtypes = [ctypes.c_uint32, P, P, ctypes.c_int, ctypes.c_int]
            lib.oracle_clique_count.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _qadj(k: int, edges) -> np.ndarray:
    a = np.zeros((k, k), dtype=np.uint8)
    for u, v in edges:
        if u == v:
            raise ValueError("query self-loop")
        a[u, v] = a[v, u] = 1
    return a


def _po_arr(po) -> np.ndarray:
    arr = np.zeros(max(2 * len(po), 2), dtype=np.int32)
    for i, (a, b) in enumerate(po):
        arr[2 * i], arr[2 * i + 1] = a, b
    return arr


def connected_order(k: int, edges, start: int = 0):
    """A matching order with connected prefixes: breadth-first from `start`, smallest id first."""
    adj = {v: set() for v in range(k)}
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    order, seen = [start], {start}
    i = 0
    while i < len(order):
        for w in sorted(adj[order[i]]):
            if w not in seen:
                seen.add(w)
                order.append(w)
        i += 1
    if len(order) != k:
        raise ValueError("query graph is not connected")
    return order


def _check(rc: int) -> int:
    if rc < 0:
        raise ValueError(f"oracle rejected its arguments (rc={rc})")
    return int(rc)


ANY_LABEL = 0xFFFFFFFF


def count(graph, k: int, edges, po=(), order=None, root_lo: int = 0, root_hi: int | None = None,
          per_root: bool = False, threads: int = 0, dlabels=None, qlabels=None):
    """Number of matches f with f(order[0]) in [root_lo, root_hi). With per_root=True returns
    (total, per-root int64 array). dlabels (n data labels) with qlabels (k query labels,
    ANY_LABEL = any) count labelled matches: label(f(v)) = qlabels[v] as well."""
    if qlabels is not None:
        return _count_labeled(graph, k, edges, po, order, root_lo, root_hi, per_root, threads, dlabels, qlabels)
    lib = _load()
    order = list(order) if order is not None else connected_order(k, edges)
    qa = _qadj(k, edges)
    oa = np.asarray(order, dtype=np.int32)
    pa = _po_arr(po)
    hi = graph.n if root_hi is None else root_hi
    pr = np.zeros(max(hi - root_lo, 1), dtype=np.int64) if per_root else None
    total = lib.oracle_count(graph.n, _ptr(graph.offsets), _ptr(graph.adj), k, _ptr(qa), _ptr(oa),
                             len(po), _ptr(pa), root_lo, hi, _ptr(pr) if pr is not None else None,
                             threads)
    total = _check(total)
    return (total, pr[: max(hi - root_lo, 0)]) if per_root else total


def _count_labeled(graph, k, edges, po, order, root_lo, root_hi, per_root, threads, dlabels, qlabels):
    lib = _load()
    order = list(order) if order is not None else connected_order(k, edges)
    qa = _qadj(k, edges)
    oa = np.asarray(order, dtype=np.int32)
    pa = _po_arr(po)
    dl = np.ascontiguousarray(dlabels, dtype=np.uint32)
    ql = np.ascontiguousarray(qlabels, dtype=np.uint32)
    if len(dl) != graph.n or len(ql) != k:
        raise ValueError("need n data labels and k query labels")
    hi = graph.n if root_hi is None else root_hi
    pr = np.zeros(max(hi - root_lo, 1), dtype=np.int64) if per_root else None
    total = _check(lib.oracle_count_labeled(graph.n, _ptr(graph.offsets), _ptr(graph.adj), _ptr(dl), k, _ptr(qa),
                                            _ptr(ql), _ptr(oa), len(po), _ptr(pa), root_lo, hi,
                                            _ptr(pr) if pr is not None else None, threads))
    return (total, pr[: max(hi - root_lo, 0)]) if per_root else total


def brute_labeled(graph, k: int, edges, dlabels, qlabels, po=()) -> int:
    """Labelled count by testing every k-tuple of distinct vertices (tiny graphs only)."""
    if graph.n ** k > 50_000_000:
        raise ValueError("brute force too large")
    lib = _load()
    qa = _qadj(k, edges)
    pa = _po_arr(po)
    dl = np.ascontiguousarray(dlabels, dtype=np.uint32)
    ql = np.ascontiguousarray(qlabels, dtype=np.uint32)
    return _check(lib.oracle_brute_labeled(graph.n, _ptr(graph.offsets), _ptr(graph.adj), _ptr(dl), k, _ptr(qa),
                                           _ptr(ql), len(po), _ptr(pa)))


def count_roots(graph, k: int, edges, roots, po=(), order=None, threads: int = 0):
    """Per-root match counts for an explicit list of roots (f(order[0]) = root)."""
    lib = _load()
    order = list(order) if order is not None else connected_order(k, edges)
    qa = _qadj(k, edges)
    oa = np.asarray(order, dtype=np.int32)
    pa = _po_arr(po)
    ra = np.ascontiguousarray(roots, dtype=np.uint32)
    out = np.zeros(max(len(ra), 1), dtype=np.int64)
    total = lib.oracle_count_roots(graph.n, _ptr(graph.offsets), _ptr(graph.adj), k, _ptr(qa),
                                   _ptr(oa), len(po), _ptr(pa), _ptr(ra), len(ra), _ptr(out), threads)
    _check(total)
    return out[: len(ra)]


def list_matches(graph, k: int, edges, po=(), order=None, cap: int | None = None) -> np.ndarray:
    """All matches as rows in query-vertex order (column v holds f(v)), sorted lexicographically."""
    lib = _load()
    order = list(order) if order is not None else connected_order(k, edges)
    qa = _qadj(k, edges)
    oa = np.asarray(order, dtype=np.int32)
    pa = _po_arr(po)
    if cap is None:
        cap = count(graph, k, edges, po, order)
    rows = np.zeros((max(cap, 1), k), dtype=np.uint32)
    total = _check(lib.oracle_list(graph.n, _ptr(graph.offsets), _ptr(graph.adj), k, _ptr(qa),
                                   _ptr(oa), len(po), _ptr(pa), _ptr(rows), cap))
    rows = rows[: min(total, cap)]
    if len(rows):
        rows = rows[np.lexsort(rows.T[::-1])]
    return rows


def brute(graph, k: int, edges, po=()) -> int:
    """Count by testing every k-tuple of distinct vertices (n**k tuples; tiny graphs only)."""
    if graph.n ** k > 50_000_000:
        raise ValueError("brute force too large")
    lib = _load()
    qa = _qadj(k, edges)
    pa = _po_arr(po)
    return _check(lib.oracle_brute(graph.n, _ptr(graph.offsets), _ptr(graph.adj), k, _ptr(qa),
                                   len(po), _ptr(pa)))


def relabel_by_degree(graph):
    """Relabel so that a smaller degree gets a smaller id (ties: smaller original id first).
    Returns (new graph, new_of_old array)."""
    from inputs import Graph

    n = graph.n
    deg = graph.degrees()
    old_of_new = np.lexsort((np.arange(n), deg))
    new_of_old = np.empty(n, dtype=np.int64)
    new_of_old[old_of_new] = np.arange(n)
    src = new_of_old[np.repeat(np.arange(n), deg)]
    dst = new_of_old[graph.adj.astype(np.int64)]
    idx = np.lexsort((dst, src))
    src, dst = src[idx], dst[idx]
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(src, minlength=n), out=offsets[1:])
    return Graph(offsets, dst.astype(np.uint32), graph.name + "-relabel"), new_of_old


def automorphisms(k: int, edges, labels=None, directed: bool = False):
    """Every vertex permutation p (p[v] is the image of v) that maps the edge set onto itself
    (with query labels: maps every vertex to one of the same label; directed: maps every arc
    u -> v to an arc p[u] -> p[v])."""
    if k > 8:
        raise ValueError("automorphism brute force limited to 8 vertices")
    es = {tuple(e) for e in edges} if directed else {frozenset(e) for e in edges}
    out = []
    for p in itertools.permutations(range(k)):
        if labels is not None and any(labels[p[v]] != labels[v] for v in range(k)):
            continue
        img = (lambda u, v: (p[u], p[v])) if directed else (lambda u, v: frozenset((p[u], p[v])))
        if all(img(u, v) in es for u, v in edges):
            out.append(p)
    return out


def symmetry_breaking_order(k: int, edges, labels=None, directed: bool = False):
    """Partial order pairs (a, b) meaning f(a) < f(b) that keep one match per automorphism
    (label-preserving automorphisms for a labelled query, arc-preserving for a directed one)."""
    group = automorphisms(k, edges, labels, directed)
    po = []
    while len(group) > 1:
        v = next(v for v in range(k) if len({p[v] for p in group}) > 1)
        orbit = sorted({p[v] for p in group})
        po.extend((v, u) for u in orbit if u != v)
        group = [p for p in group if p[v] == v]
    return po


def prefix_counts(graph, k: int, edges, order, po=(), threads: int = 0):
    """|R(q'_i)| for i = 1..k, q'_i the sub-query induced by order[:i] with its own PO pairs."""
    out = []
    for i in range(1, k + 1):
        vs = list(order[:i])
        idx = {v: j for j, v in enumerate(vs)}
        sub_e = [(idx[u], idx[v]) for u, v in edges if u in idx and v in idx]
        sub_po = [(idx[a], idx[b]) for a, b in po if a in idx and b in idx]
        if i == 1:
            out.append(graph.n)
            continue
        out.append(count(graph, i, sub_e, sub_po, order=list(range(i)), threads=threads))
    return out


def motif_key(k: int, edges) -> int:
    """Isomorphism-class key of a graph on k vertices: the smallest adjacency bitmask (bit
    i * k + j for every edge {i, j}, both directions) over all relabellings."""
    best = None
    for p in itertools.permutations(range(k)):
        m = 0
        for u, v in edges:
            a, b = p[u], p[v]
            m |= (1 << (a * k + b)) | (1 << (b * k + a))
        best = m if best is None else min(best, m)
    return best


def motif_census(graph, k: int):
    """Induced motif census by definition: every k-vertex subset of the (tiny) graph whose
    induced subgraph is connected, counted per isomorphism class ({motif_key: count})."""
    off = graph.offsets.astype(np.int64)
    nbr = [set(map(int, graph.adj[off[u]:off[u + 1]])) for u in range(graph.n)]
    out = {}
    for vs in itertools.combinations(range(graph.n), k):
        es = [(i, j) for i in range(k) for j in range(i + 1, k) if vs[j] in nbr[vs[i]]]
        seen, todo = {0}, [0]
        while todo:
            u = todo.pop()
            for i, j in es:
                w = j if i == u else i if j == u else None
                if w is not None and w not in seen:
                    seen.add(w)
                    todo.append(w)
        if len(seen) == k:
            key = motif_key(k, es)
            out[key] = out.get(key, 0) + 1
    return out


def walk_traces(graph, threads: int = 0):
    """(tr(A^3), tr(A^4)) of the graph's adjacency matrix, by sparse 2-walk counting."""
    lib = _load()
    out = np.zeros(2, dtype=np.uint64)
    rc = lib.oracle_walk_traces(graph.n, _ptr(graph.offsets), _ptr(graph.adj), threads, _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_walk_traces could not allocate its counters")
    return int(out[0]), int(out[1])


def triangle_count_trace(graph, threads: int = 0) -> int:
    """#K3 = tr(A^3) / 6."""
    t3, _ = walk_traces(graph, threads)
    if t3 % 6:
        raise ArithmeticError("tr(A^3) is not a multiple of 6: the graph is not simple")
    return t3 // 6


def c4_count_trace(graph, threads: int = 0) -> int:
    """#C4 = (tr(A^4) - 2m - 4 sum_v C(d(v), 2)) / 8, in exact integers."""
    _, t4 = walk_traces(graph, threads)
    d = graph.degrees().astype(object)
    rest = t4 - 2 * graph.m - 4 * int(sum(x * (x - 1) // 2 for x in d.tolist()))
    if rest % 8 or rest < 0:
        raise ArithmeticError("closed 4-walk count inconsistent with a simple graph")
    return rest // 8


def clique_count(graph, k: int, threads: int = 0) -> int:
    """Number of k-vertex cliques (degree-orientation method, independent of the backtracker)."""
    lib = _load()
    return _check(lib.oracle_clique_count(graph.n, _ptr(graph.offsets), _ptr(graph.adj), k, threads))


def reverse_csr(graph):
    """In-lists of a directed graph given by its out-lists (the CSR of the reversed arcs)."""
    from inputs import Graph

    n = graph.n
    src = np.repeat(np.arange(n, dtype=np.int64), graph.degrees())
    dst = graph.adj.astype(np.int64)
    idx = np.lexsort((src, dst))
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(dst, minlength=n), out=offsets[1:])
    return Graph(offsets, src[idx].astype(np.uint32), graph.name + "-reversed")


def _labels_pair(graph, k, dlabels, qlabels):
    """Both label arrays (uint32, n and k entries) or neither."""
    if (dlabels is None) != (qlabels is None):
        raise ValueError("give data and query labels together")
    if dlabels is None:
        return None, None
    dl = np.ascontiguousarray(dlabels, dtype=np.uint32)
    ql = np.ascontiguousarray(qlabels, dtype=np.uint32)
    if len(dl) != graph.n or len(ql) != k:
        raise ValueError("need n data labels and k query labels")
    return dl, ql


def count_directed(graph, k: int, arcs, po=(), order=None, root_lo: int = 0, root_hi: int | None = None,
                   threads: int = 0, dlabels=None, qlabels=None):
    """Matches of a directed query (arcs (a, b) meaning a -> b) in a directed graph given by its
    out-lists: every query arc must map to a data arc. dlabels / qlabels as in ``count``."""
    lib = _load()
    dl, ql = _labels_pair(graph, k, dlabels, qlabels)
    order = list(order) if order is not None else connected_order(k, arcs)
    qa = np.zeros((k, k), dtype=np.uint8)
    for a, b in arcs:
        if a == b:
            raise ValueError("query self-loop")
        qa[a, b] = 1
    rg = reverse_csr(graph)
    oa = np.asarray(order, dtype=np.int32)
    pa = _po_arr(po)
    hi = graph.n if root_hi is None else root_hi
    return _check(lib.oracle_count_directed(graph.n, _ptr(graph.offsets), _ptr(graph.adj), _ptr(rg.offsets),
                                            _ptr(rg.adj), _ptr(dl) if dl is not None else None, k, _ptr(qa),
                                            _ptr(ql) if ql is not None else None, _ptr(oa), len(po), _ptr(pa),
                                            root_lo, hi, None, threads))


def brute_directed(graph, k: int, arcs, po=(), dlabels=None, qlabels=None) -> int:
    """Directed count by testing every k-tuple of distinct vertices (tiny graphs only)."""
    if graph.n ** k > 50_000_000:
        raise ValueError("brute force too large")
    lib = _load()
    dl, ql = _labels_pair(graph, k, dlabels, qlabels)
    qa = np.zeros((k, k), dtype=np.uint8)
    for a, b in arcs:
        qa[a, b] = 1
    pa = _po_arr(po)
    return _check(lib.oracle_brute_directed(graph.n, _ptr(graph.offsets), _ptr(graph.adj),
                                            _ptr(dl) if dl is not None else None, k, _ptr(qa),
                                            _ptr(ql) if ql is not None else None, len(po), _ptr(pa)))
