"""Parity at the workloads' full sizes, in the launch configuration the benchmark times:
per-root counts on stratified root samples (the heaviest hubs included) against the oracle,
which computes them one root at a time."""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


def _roots(gr, s, seed):
    n = gr.n
    rng = np.random.default_rng(seed)
    r = (np.arange(s) * (n // s) + rng.integers(0, n // s, s)).astype(np.uint32)
    hubs = np.argsort(gr.degrees())[-6:].astype(np.uint32)
    return np.unique(np.concatenate([r, hubs]))


def _check(huge, G, gr, names, s, seed):
    for name in names:
        k, e = inputs.QUERIES[name]
        p = huge.Plan(G, k, e)  # plan of Alg. 1, as in the benchmark
        d = p.describe()
        assert d["op"] == "EXTEND-CHAIN"
        order = d["chain"]["order"]
        po = [tuple(x) for x in d["po"]]
        roots = _roots(gr, s, seed)
        want = oracle.count_roots(gr, k, e, roots, po, order)
        got = [huge.enumerate(p, roots=[int(r)], mem_bound=8 << 30) for r in roots]
        assert got == list(map(int, want)), name


def test_rmat20_k4_c4_sampled_roots(gpu_lib):
    g = inputs.workload_graph("rmat20")
    gr, _ = oracle.relabel_by_degree(g)
    G = gpu_lib.Graph(g.offsets, g.adj)
    _check(gpu_lib, G, gr, ["k4", "c4"], 40, 20)


def test_chunglu_5vertex_sampled_roots(gpu_lib):
    g = inputs.workload_graph("chunglu4m")
    gr, _ = oracle.relabel_by_degree(g)
    G = gpu_lib.Graph(g.offsets, g.adj)
    _check(gpu_lib, G, gr, ["k5", "house", "tailed_diamond_a"], 24, 30)
