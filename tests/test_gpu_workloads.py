"""Parity at the workloads' full sizes, in the launch configuration the benchmark times:
per-root counts on stratified root samples (the heaviest hubs included) against the oracle,
which computes them one root at a time."""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


def _roots(gr, s, seed, hubs=True):
    n = gr.n
    rng = np.random.default_rng(seed)
    r = (np.arange(s) * (n // s) + rng.integers(0, n // s, s)).astype(np.uint32)
    if not hubs:
        return np.unique(r)
    top = np.argsort(gr.degrees())[-6:].astype(np.uint32)
    return np.unique(np.concatenate([r, top]))


def _check(huge, G, gr, names, s, seed, hubs_for=(), given_order=False):
    from paper_2103_14294_b300.experiments import _order

    for name in names:
        k, e = inputs.QUERIES[name]
        po = oracle.symmetry_breaking_order(k, e)
        if given_order:
            p = huge.Plan(G, k, e, order=_order(k, e, po), po=po)
        else:
            p = huge.Plan(G, k, e, po=po)  # plan of Alg. 1, as in the benchmark
        d = p.describe()
        assert d["op"] == "EXTEND-CHAIN"
        order = d["chain"]["order"]
        roots = _roots(gr, s, seed, hubs=name in hubs_for)
        want = oracle.count_roots(gr, k, e, roots, po, order)
        got = [huge.enumerate(p, roots=[int(r)], mem_bound=8 << 30) for r in roots]
        assert got == list(map(int, want)), name


def test_rmat20_k4_c4_sampled_roots(gpu_lib):
    """The benchmark workload and plans: 40 stratified roots plus the 6 largest hubs."""
    g = inputs.workload_graph("rmat20")
    gr, _ = oracle.relabel_by_degree(g)
    G = gpu_lib.Graph(g.offsets, g.adj)
    _check(gpu_lib, G, gr, ["k4", "c4"], 40, 20, hubs_for=("k4", "c4"))


def test_chunglu_5vertex_sampled_roots(gpu_lib):
    """Chung-Lu 4M/35M: 24 stratified roots (the oracle's plain backtracking cannot finish the
    house or the tailed diamond from the hubs); the 6 largest hubs as roots for the 5-clique."""
    g = inputs.workload_graph("chunglu4m")
    gr, _ = oracle.relabel_by_degree(g)
    G = gpu_lib.Graph(g.offsets, g.adj)
    _check(gpu_lib, G, gr, ["k5", "house", "tailed_diamond_a"], 24, 30, hubs_for=("k5",), given_order=True)


def test_root_range_shards_add_up_to_the_whole_count(gpu_lib):
    """The multi-GPU split run on one GPU: the library's root-range launches over the ranges of
    shard.shard_bounds (computed on the relabelled degree sequence) add up to the whole count,
    for 2, 3 and 5 ranks."""
    from paper_2103_14294_b300 import shard

    huge = gpu_lib
    g = inputs.rmat(13, 8, 71)
    gr, _ = oracle.relabel_by_degree(g)
    G = huge.Graph(g.offsets, g.adj)
    off = shard.relabelled_offsets(g)
    assert np.array_equal(off, gr.offsets.astype(np.int64))
    for name in ("triangle", "c4", "tailed_triangle"):
        k, e = inputs.QUERIES[name]
        po = oracle.symmetry_breaking_order(k, e)
        want = oracle.count(gr, k, e, po)
        p = huge.Plan(G, k, e, po=po, flags=huge.PLAN_EXTEND_ONLY)  # root ranges need an EXTEND chain
        for world in (2, 3, 5):
            parts = [huge.enumerate(p, root_range=shard.shard_of(off, r, world)) for r in range(world)]
            assert sum(parts) == want, (name, world, parts)
