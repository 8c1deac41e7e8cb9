"""The allocation-free entry point (huge_count_noalloc) against the oracle and the regular one.

huge_count_noalloc exists for callers that cannot allocate device memory (their memory is owned
by another allocator or a fixed budget); it keeps its scratch in a static device array. The
paper has no counterpart to it. This file is collected last so that a failure here does not
hide any other test's result; it also passes when run alone.
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


def _device_csr(g):
    import torch

    d_off = torch.from_numpy(g.offsets.astype(np.uint32).view(np.int32)).cuda()
    d_adj = torch.from_numpy(g.adj.view(np.int32)).cuda()
    return d_off, d_adj


def test_noalloc_matches_oracle_and_huge_enumerate_twice(gpu_lib):
    import torch

    huge = gpu_lib
    g = inputs.rmat(10, 8, 77)
    G = huge.Graph(g.offsets, g.adj, flags=0)  # same ids on both paths: no relabelling
    d_off, d_adj = _device_csr(g)
    # the oracle counts on the degree-relabelled copy (fast: low-degree roots first); with a
    # complete symmetry-breaking order, or none, the count does not depend on the ids
    gr = oracle.relabel_by_degree(g)[0]
    for name in ["triangle", "k4", "c4", "house", "tailed_diamond_a"]:
        k, e = inputs.QUERIES[name]
        po = oracle.symmetry_breaking_order(k, e)
        want = oracle.count(gr, k, e, po)
        order = oracle.connected_order(k, e)
        assert huge.enumerate(huge.Plan(G, k, e, order=order)) == want, name
        for _ in range(2):  # the static scratch keeps the previous call's contents
            assert huge.count_noalloc(d_off, d_adj, g.n, g.nnz, k, e, order=order) == want, name
        # the library-chosen order, and an explicit partial order
        assert huge.count_noalloc(d_off, d_adj, g.n, g.nnz, k, e) == want, name
        assert huge.count_noalloc(d_off, d_adj, g.n, g.nnz, k, e, order=order, po=po) == want, name
    k, e = inputs.QUERIES["c4"]
    assert huge.count_noalloc(d_off, d_adj, g.n, g.nnz, k, e, po=[]) == oracle.count(gr, k, e, [])
    torch.cuda.synchronize()


def test_noalloc_rejects_bad_arguments(gpu_lib):
    import torch

    huge = gpu_lib
    g = inputs.er(50, 100, 5)
    d_off, d_adj = _device_csr(g)
    k = huge.MAX_QUERY_VERTICES + 1
    edges = [(i, i + 1) for i in range(k - 1)]
    with pytest.raises(huge.HugeError) as ei:
        huge.count_noalloc(d_off, d_adj, g.n, g.nnz, k, edges)
    assert ei.value.code == huge.EINVAL
    tri = inputs.QUERIES["triangle"][1]
    for bad in (dict(nnz=1 << 32), dict(n=g.n + 5), dict(nnz=g.nnz + 1)):
        args = dict(n=g.n, nnz=g.nnz)
        args.update(bad)
        with pytest.raises(huge.HugeError) as ei:
            huge.count_noalloc(d_off, d_adj, args["n"], args["nnz"], 3, tri)
        assert ei.value.code == huge.EINVAL
    with pytest.raises(huge.HugeError):  # wrong dtype
        huge.count_noalloc(d_off.to(torch.int64), d_adj, g.n, g.nnz, 3, tri)
    with pytest.raises(huge.HugeError):  # host tensor
        huge.count_noalloc(d_off.cpu(), d_adj, g.n, g.nnz, 3, tri)
