"""The CSR contract of huge_graph_load, checked on the host before any device memory is touched
(so these tests need no GPU): malformed graphs fail with HUGE_EINVAL and a message naming the
fault; well-formed ones pass validation. On a machine without a GPU, a graph that passes
validation then fails its device allocation with HUGE_ENOMEM, never with HUGE_EINVAL.
"""
import numpy as np
import pytest

import inputs
from paper_2103_14294_b300 import huge


def _csr(lists):
    off = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.uint64)
    adj = np.asarray([v for x in lists for v in x], dtype=np.uint32)
    return off, adj


def _load(off, adj, **kw):
    """None if the graph passed validation (loaded, or only its device allocation failed),
    else the HugeError."""
    try:
        huge.Graph(off, adj, **kw).handle
    except huge.HugeError as e:
        if e.code == huge.ENOMEM:
            return None
        return e
    return None


TRIANGLE = [[1, 2], [0, 2], [0, 1]]


@pytest.mark.parametrize("lists,why", [
    ([[2, 1], [0, 2], [0, 1]], "not strictly increasing"),  # unsorted
    ([[1, 1, 2], [0, 2], [0, 1]], "not strictly increasing"),  # duplicate
    ([[0, 1, 2], [0, 2], [0, 1]], "self-loop"),
    ([[1, 2], [0, 2], [0, 1, 3]], "neighbour id >= n"),
    ([[1, 2], [0], [0, 1]], "not symmetric"),  # 1 -> 2 has no mirror
    ([[1], [0, 2], [0, 1]], "not symmetric"),  # 2 -> 0 has no mirror
])
def test_malformed_undirected_csr_is_rejected(lists, why):
    off, adj = _csr(lists)
    err = _load(off, adj)
    assert err is not None and err.code == huge.EINVAL and why in str(err), (lists, err)


def test_malformed_offsets_and_sizes_are_rejected():
    off, adj = _csr(TRIANGLE)
    bad = off.copy()
    bad[0] = 1
    assert _load(bad, adj).code == huge.EINVAL
    bad = off.copy()
    bad[1], bad[2] = bad[2], bad[1]  # decreasing
    assert _load(bad, adj).code == huge.EINVAL
    assert _load(np.zeros(1, dtype=np.uint64), np.zeros(0, dtype=np.uint32)).code == huge.EINVAL  # n = 0


def test_binding_checks_array_lengths_before_the_call():
    """The C ABI takes plain pointers; the binding refuses arrays shorter than what the library
    would read (offsets[0..n], adj[0..offsets[n]), n labels)."""
    off, adj = _csr(TRIANGLE)
    for args, kw in [((off, adj[:-1]), {}), ((off[:-1], adj), {"n": 3}), ((off, adj), {"n": 4}),
                     ((off, adj), {"labels": np.zeros(2, dtype=np.uint32), "nlabels": 1})]:
        with pytest.raises(huge.HugeError) as ei:
            huge.Graph(*args, **kw)
        assert ei.value.code == huge.EINVAL


def test_labels_must_lie_below_nlabels():
    off, adj = _csr(TRIANGLE)
    assert _load(off, adj, labels=np.array([0, 1, 2], dtype=np.uint32), nlabels=2).code == huge.EINVAL
    assert _load(off, adj, labels=np.array([0, 1, 1], dtype=np.uint32), nlabels=2) is None


def test_well_formed_graphs_pass_validation():
    off, adj = _csr(TRIANGLE)
    assert _load(off, adj) is None
    assert _load(*_csr([[], [], []])) is None  # isolated vertices only
    for g in (inputs.er(200, 900, 3), inputs.rmat(10, 8, 4), inputs.complete(9)):
        assert _load(g.offsets, g.adj) is None
    # a directed graph needs no mirror arcs
    d = inputs.gnp_directed(30, 1, 4, 2)
    assert _load(d.offsets, d.adj, flags=huge.RELABEL_BY_DEGREE | huge.DIRECTED) is None
    off, adj = _csr([[1, 2], [2], []])
    assert _load(off, adj, flags=huge.DIRECTED) is None
    assert _load(off, adj).code == huge.EINVAL  # the same arcs read as an undirected graph


def test_every_single_entry_removal_or_insertion_breaks_symmetry():
    """Drop one entry, or add one (keeping the list sorted), anywhere in a random graph: the
    mirror is missing and validation says so, whether the broken entry points up or down."""
    g = inputs.gnp(30, 1, 4, 12)
    lists = [list(map(int, g.adj[g.offsets[v]:g.offsets[v + 1]])) for v in range(g.n)]
    rng = np.random.default_rng(0)
    for _ in range(60):
        ls = [list(x) for x in lists]
        v = int(rng.integers(g.n))
        if rng.random() < 0.5 and ls[v]:
            ls[v].pop(int(rng.integers(len(ls[v]))))
        else:
            free = [u for u in range(g.n) if u != v and u not in ls[v]]
            ls[v] = sorted(ls[v] + [int(rng.choice(free))])
        err = _load(*_csr(ls))
        assert err is not None and err.code == huge.EINVAL and "not symmetric" in str(err)
