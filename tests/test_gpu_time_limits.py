"""Failure paths on the GPU, made without a fault. A launch whose time limit passes returns
HUGE_ETIMEOUT: its warps see the limit on the device clock, leave their loops and raise a flag
that the host reads. The next calls on the same graph and device then give exact counts again.
"""
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu
Q = inputs.QUERIES


def test_time_limit_returns_etimeout_and_the_context_stays_usable(gpu_lib):
    huge = gpu_lib
    g = inputs.rmat(18, 16, 9)  # its 4-cycles take about a hundred times longer than 1 ms
    G = huge.Graph(g.offsets, g.adj)
    k, e = Q["c4"]
    po4 = oracle.symmetry_breaking_order(k, e)
    heavy = huge.Plan(G, k, e, order=[0, 1, 3, 2], po=po4)
    with pytest.raises(huge.HugeError) as ei:
        huge.enumerate(heavy, time_limit_ms=1)
    assert ei.value.code == huge.ETIMEOUT
    with pytest.raises(huge.HugeError) as ei:
        huge.enumerate_batch([heavy, heavy], time_limit_ms=1)
    assert ei.value.code == huge.ETIMEOUT
    # the same graph, plan and device serve the next calls exactly (whole-graph counts from
    # closed walks of the adjacency matrix: no enumeration on the oracle side)
    k3, tri = Q["triangle"]
    small = huge.Plan(G, k3, tri, order=[0, 1, 2], po=oracle.symmetry_breaking_order(k3, tri))
    assert huge.enumerate(small) == oracle.triangle_count_trace(g)
    assert huge.enumerate(heavy) == oracle.c4_count_trace(g)
