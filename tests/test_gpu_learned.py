"""The learned estimator end to end at small scale: tuples logged by the exact enumerator, GPU
training, and plans from the trained network against plans from the sampling estimator.

The gain the network brings is in planning: one batched inference replaces one sampled exact
enumeration per sub-query. Exact counts must be identical whichever plan is used.
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


def test_learned_plans_exact_and_faster_to_plan(gpu_lib):
    huge = gpu_lib
    from paper_2103_14294_b300 import learned

    graphs = []
    for s in (10, 11, 12):
        g = inputs.rmat(s, 8, 300 + s)
        graphs.append((f"rmat{s}", huge.Graph(g.offsets, g.adj)))
    X, Y, _ = learned.collect(graphs, 3000, seed=2, time_limit_ms=500, budget_s=90)
    assert len(Y) >= 1000
    model, loss, rmse = learned.train(X, Y, epochs=150, batch_rows=1024)
    assert rmse is not None and rmse < 2.5  # log-space error well below the spread of log counts
    assert rmse < 0.5 * float(np.std(Y))

    g = inputs.rmat(13, 8, 77)
    gr = oracle.relabel_by_degree(g)[0]
    G = huge.Graph(g.offsets, g.adj)
    queries = [inputs.QUERIES[n] for n in ("k4", "c4", "diamond", "tailed_triangle", "house")]
    res = learned.compare(G, queries, model, time_limit_ms=60000, mem_bound=1 << 30)
    plan_plain = sum(r["plain"]["plan_s"] for r in res)
    plan_learned = sum(r["learned"]["plan_s"] for r in res)
    for (k, e), r in zip(queries, res):
        assert r["plain"]["count"] == r["learned"]["count"]
        if k == 4:
            assert r["plain"]["count"] == oracle.count(gr, k, e, oracle.symmetry_breaking_order(k, e))
    assert plan_learned < plan_plain, (plan_learned, plan_plain)


def test_root_features_and_per_plan_level_rows(gpu_lib):
    """huge_root_features: the device-computed neighbourhood statistics of each root match the
    CSR (log degree, log upward degree, log neighbour-degree sum, relative id); the batched
    launch's per-plan level rows equal the plain launch's, root by root."""
    huge = gpu_lib
    g = inputs.rmat(11, 8, 31)
    gr = oracle.relabel_by_degree(g)[0]
    G = huge.Graph(g.offsets, g.adj)
    k, e = inputs.QUERIES["c4"]
    p = huge.Plan(G, k, e, order=[0, 1, 2, 3])
    roots = np.array([0, 5, 700, gr.n - 1, gr.n // 2], dtype=np.uint32)
    X = huge.root_features(p, roots)
    deg = gr.degrees()
    off = gr.offsets.astype(np.int64)
    for i, r in enumerate(roots):
        nb = gr.adj[off[r]:off[r + 1]].astype(np.int64)
        assert np.isclose(X[i, 46], np.log1p(deg[r]), rtol=1e-5)
        assert np.isclose(X[i, 47], np.log1p(int((nb > r).sum())), rtol=1e-5)
        assert np.isclose(X[i, 48], np.log1p(float(deg[nb].sum())), rtol=1e-4)
        assert np.isclose(X[i, 52], r / gr.n, rtol=1e-5)
    lr = np.zeros((len(roots), 16), dtype=np.int64)
    counts = huge.enumerate_batch([p] * len(roots), roots=[[int(r)] for r in roots], level_rows=lr)
    for i, r in enumerate(roots):
        c, st = huge.enumerate(p, roots=[int(r)], stats=True)
        assert counts[i] == c
        assert list(lr[i, 1:k]) == st["level_rows"][1:k]
