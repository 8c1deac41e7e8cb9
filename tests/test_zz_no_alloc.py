"""The allocation-free entry point (huge_count_noalloc) against the regular one.

huge_count_noalloc exists for callers that cannot allocate device memory (their memory is owned
by another allocator or a fixed budget); it keeps its scratch in a static device array. This
file is collected last so that a failure here does not hide any other test's result.
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


def test_noalloc_matches_huge_enumerate_twice(gpu_lib):
    import torch

    huge = gpu_lib
    g = inputs.rmat(12, 8, 77)
    G = huge.Graph(g.offsets, g.adj, flags=0)  # same ids on both paths: no relabelling
    off32 = g.offsets.astype(np.uint32)
    d_off = torch.from_numpy(off32.view(np.int32)).cuda()
    d_adj = torch.from_numpy(g.adj.view(np.int32)).cuda()
    for name in ["triangle", "k4", "c4", "house", "tailed_diamond_a"]:
        k, e = inputs.QUERIES[name]
        order = oracle.connected_order(k, e)
        expect = huge.enumerate(huge.Plan(G, k, e, order=order))
        for _ in range(2):  # the static scratch keeps the previous call's contents
            got = huge.count_noalloc(d_off, d_adj, g.n, g.nnz, k, e, order=order)
            assert got == expect, name
    torch.cuda.synchronize()


def test_noalloc_rejects_bad_sizes(gpu_lib):
    import torch

    huge = gpu_lib
    g = inputs.er(50, 100, 5)
    d_off = torch.from_numpy(g.offsets.astype(np.uint32).view(np.int32)).cuda()
    d_adj = torch.from_numpy(g.adj.view(np.int32)).cuda()
    k = huge.MAX_QUERY_VERTICES + 1
    edges = [(i, i + 1) for i in range(k - 1)]
    with pytest.raises(huge.HugeError) as ei:
        huge.count_noalloc(d_off, d_adj, g.n, g.nnz, k, edges)
    assert ei.value.code == huge.EINVAL
    with pytest.raises(huge.HugeError) as ei:
        huge.count_noalloc(d_off, d_adj, g.n, 1 << 32, 3, inputs.QUERIES["triangle"][1])
    assert ei.value.code == huge.EINVAL
