"""Out-of-core adjacency (huge_graph_set_residency): with only part of the adjacency array in
HBM and the rest read from host memory, every count stays the oracle's."""
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


def test_residency_budgets_keep_counts_exact(gpu_lib):
    huge = gpu_lib
    g = inputs.rmat(13, 8, 91)
    gr, _ = oracle.relabel_by_degree(g)
    G = huge.Graph(g.offsets, g.adj)
    adj_bytes = ((g.nnz + 3) // 4 * 4 + 4) * 4
    want = {}
    for name in ("triangle", "c4", "k4", "diamond"):
        k, e = inputs.QUERIES[name]
        want[name] = oracle.count(gr, k, e, oracle.symmetry_breaking_order(k, e))
    for budget in (0, 2 << 20, adj_bytes // 2, 1 << 62):
        resident = G.set_residency(budget)
        assert resident <= max(budget, 0) or budget >= adj_bytes
        if budget == 0:
            assert resident == 0
        for name, w in want.items():
            k, e = inputs.QUERIES[name]
            assert huge.enumerate(huge.Plan(G, k, e)) == w, (name, budget)
    # hub bitmaps rebuilt from the managed array, and LIST from host-resident lists
    G.set_residency(0)
    G.set_hub_bitmaps(64, 1 << 30)
    k, e = inputs.QUERIES["c4"]
    assert huge.enumerate(huge.Plan(G, k, e)) == want["c4"]
