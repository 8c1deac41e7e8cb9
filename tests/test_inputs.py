"""The seeded input generators against their recipes: every graph is a simple CSR (sorted,
no loops, no repeats; symmetric unless directed), sizes are the ones the recipes state, the
output depends only on the seed (not on the host's thread count), and random queries are
connected simple graphs."""
import hashlib
import os
import subprocess
import sys

import numpy as np
import pytest

import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _check_csr(g, symmetric=True):
    off = np.asarray(g.offsets, dtype=np.int64)
    adj = np.asarray(g.adj, dtype=np.int64)
    assert off[0] == 0 and off[-1] == len(adj) and np.all(np.diff(off) >= 0)
    src = np.repeat(np.arange(g.n), np.diff(off))
    assert np.all(adj < g.n) and not np.any(adj == src)  # ids in range, no self-loops
    same_row = src[1:] == src[:-1]
    assert np.all(adj[1:][same_row] > adj[:-1][same_row])  # strictly increasing lists
    if symmetric:
        fwd = np.sort(src * g.n + adj)
        rev = np.sort(adj * g.n + src)
        assert np.array_equal(fwd, rev)
    return src, adj


@pytest.mark.parametrize("make,symmetric", [
    (lambda: inputs.er(500, 3000, 1), True),
    (lambda: inputs.gnp(60, 1, 5, 2), True),
    (lambda: inputs.rmat(12, 16, 3), True),
    (lambda: inputs.chung_lu(8192, 40000, 4, max_w=300.0), True),
    (lambda: inputs.complete(7), True),
    (lambda: inputs.complete_bipartite(3, 5), True),
    (lambda: inputs.rmat_directed(11, 8, 5), False),
    (lambda: inputs.gnp_directed(50, 1, 4, 6), False),
])
def test_graphs_are_simple_csr(make, symmetric):
    _check_csr(make(), symmetric)


def test_recipe_sizes():
    assert inputs.er(2000, 20000, 1).nnz == 2 * 20000  # exactly m distinct pairs
    g = inputs.workload_graph("chunglu64k")
    assert g.n == 65536 and g.nnz == 2 * 546_875  # exactly m distinct edges
    deg = np.diff(np.asarray(g.offsets, dtype=np.int64))
    assert 350 < deg.max() < 1400  # hubs near the maximum weight (700)
    assert inputs.complete(9).nnz == 9 * 8 and inputs.complete_bipartite(3, 5).nnz == 2 * 15
    r = inputs.rmat(10, 8, 7)
    assert r.n == 1024 and r.nnz <= 2 * 8 * 1024  # repeats and loops only ever removed


def test_rmat_is_skewed_and_er_is_not():
    """R-MAT (a = 0.57) concentrates edges on few vertices; G(n, m) does not."""
    r = np.diff(np.asarray(inputs.rmat(14, 16, 2).offsets, dtype=np.int64))
    e = np.diff(np.asarray(inputs.er(1 << 14, int(r.sum() // 2), 2).offsets, dtype=np.int64))
    assert r.max() > 20 * r.mean() and e.max() < 4 * e.mean()


def test_same_seed_same_graph_other_seed_other_graph():
    a, b, c = inputs.rmat(11, 8, 9), inputs.rmat(11, 8, 9), inputs.rmat(11, 8, 10)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.adj, b.adj)
    assert not (len(a.adj) == len(c.adj) and np.array_equal(a.adj, c.adj))


_DIGEST = """
import hashlib, sys
sys.path.insert(0, {root!r})
import inputs
h = hashlib.sha256()
for g in (inputs.rmat(13, 16, 2), inputs.chung_lu(1 << 14, 90000, 3, max_w=500.0), inputs.er(3000, 20000, 1)):
    h.update(g.offsets.tobytes()); h.update(g.adj.tobytes())
print(h.hexdigest())
"""


def test_output_does_not_depend_on_the_thread_count():
    digests = set()
    for threads in ("1", "3", str(os.cpu_count() or 4)):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        out = subprocess.run([sys.executable, "-c", _DIGEST.format(root=ROOT)], env=env, check=True,
                             capture_output=True, text=True).stdout.strip()
        digests.add(out)
    assert len(digests) == 1, digests


def test_random_queries_are_connected_simple_graphs():
    for k in range(2, 9):
        for seed in range(20):
            kk, e = inputs.random_query(k, 1000 * k + seed)
            assert kk == k
            es = {frozenset(x) for x in e}
            assert len(es) == len(e) and all(len(x) == 2 for x in es)  # no repeats, no loops
            assert all(0 <= u < k for x in e for u in x)
            seen, todo = {0}, [0]
            while todo:
                u = todo.pop()
                for x in es:
                    if u in x:
                        (v,) = x - {u}
                        if v not in seen:
                            seen.add(v)
                            todo.append(v)
            assert len(seen) == k  # connected: a spanning tree is always drawn
            assert len(e) >= k - 1
    # every extra pair with probability 1: the complete graph
    assert len(inputs.random_query(6, 5, 1, 1)[1]) == 15


def test_uniform_draws_lie_in_range_and_cover_it():
    x = inputs.uniform(20000, 7, 3)
    assert x.min() == 0 and x.max() == 6
    counts = np.bincount(x.astype(np.int64), minlength=7)
    assert counts.min() > 0.8 * 20000 / 7
    assert np.array_equal(x, inputs.uniform(20000, 7, 3))
