"""Host logic of the learned-estimator pipeline (no GPU): how batched exact runs become
training tuples, and the matching orders used to log them.

A training tuple pairs a sub-query q' with log(1 + |R(q')|). There is one tuple for every
prefix of three or more vertices of an EXTEND chain's matching order. The library's batched
launch reports the rows after each operator and the count. These tests stand a fake in for
the library's batched call, so what they check is the bookkeeping:

* which prefix each value belongs to;
* how a batch that hits its time limit is split. The runs that fit are kept; a lone run that
  does not fit is dropped.
"""
import math
import types

import numpy as np
import pytest

import inputs
from paper_2103_14294_b300 import huge as real_huge
from paper_2103_14294_b300 import learned


class _Edges(list):
    """A query's edge list that also carries the item's position in the batch."""

    def __init__(self, edges, pos):
        super().__init__(edges)
        self.pos = pos


class _FakeHuge:
    """The two library calls _batch_tuples makes. A plan's level i (after the SCAN) has
    10 ** i + k rows and its count is 10 ** (k - 1) + 7; a batch holding an item whose position
    is in `slow` raises HUGE_ETIMEOUT, as a launch that reaches its time limit does."""
    HugeError = real_huge.HugeError
    ETIMEOUT, EOVERFLOW = real_huge.ETIMEOUT, real_huge.EOVERFLOW

    def __init__(self, slow=()):
        self.slow = set(slow)
        self.calls = []

    def Plan(self, G, k, e, order=None):
        return types.SimpleNamespace(k=k, pos=getattr(e, "pos", None), free=lambda: None)

    def enumerate_batch(self, plans, level_rows=None, time_limit_ms=None, mem_bound=None):
        self.calls.append([p.pos for p in plans])
        if any(p.pos in self.slow for p in plans):
            raise real_huge.HugeError(real_huge.ETIMEOUT, "time limit")
        for q, p in enumerate(plans):
            for i in range(p.k):
                level_rows[q, i] = 10 ** i + p.k
        return [10 ** (p.k - 1) + 7 for p in plans]


def _batch_tuples(fake, items):
    orig = learned.huge
    learned.huge = fake
    try:
        out = []
        learned._batch_tuples(None, items, 50, 1 << 30, out)
        return out
    finally:
        learned.huge = orig


def test_batch_tuples_map_level_rows_to_prefixes():
    items = [(3, [(0, 1), (1, 2)], [1, 0, 2]), (5, inputs.QUERIES["house"][1], [0, 1, 4, 2, 3])]
    out = _batch_tuples(_FakeHuge(), items)
    assert len(out) == 1 + 3  # k - 2 prefixes per query
    k, _, mask, y = out[0]
    assert (k, mask) == (3, 0b111) and y == pytest.approx(math.log1p(10 ** 2 + 7))  # the count
    house = [(m, y) for kk, _, m, y in out if kk == 5]
    assert [m for m, _ in house] == [0b10011, 0b10111, 0b11111]  # {0, 1, 4}, then + 2, + 3
    assert house[0][1] == pytest.approx(math.log1p(10 ** 2 + 5))  # rows after the 3rd vertex
    assert house[1][1] == pytest.approx(math.log1p(10 ** 3 + 5))
    assert house[2][1] == pytest.approx(math.log1p(10 ** 4 + 7))  # the last prefix: the count


@pytest.mark.parametrize("slow", [set(), {3}, {3, 11}, {0, 1, 2, 3, 4, 5, 6, 7}, set(range(16))])
def test_batch_tuples_split_timed_out_batches_and_drop_only_the_slow_runs(slow):
    tri = inputs.QUERIES["triangle"][1]
    items = [(3, _Edges(tri, i), [0, 1, 2]) for i in range(16)]
    fake = _FakeHuge(slow)
    out = _batch_tuples(fake, items)
    assert sorted(e.pos for _, e, _, _ in out) == sorted(set(range(16)) - slow)
    # every run that fits was part of exactly one launch that finished
    done = [p for c in fake.calls if not set(c) & slow for p in c]
    assert sorted(done) == sorted(set(range(16)) - slow)
    # binary splitting: a slow run is in at most log2(16) + 1 = 5 failed launches
    failed = [c for c in fake.calls if set(c) & slow]
    assert all(sum(s in c for c in failed) <= 5 for s in slow)
    assert len(failed) <= 31  # 1 + 2 + 4 + 8 + 16 launches when every run is slow


def test_batch_tuples_reraise_other_errors():
    class _Broken(_FakeHuge):
        def enumerate_batch(self, plans, **kw):
            raise real_huge.HugeError(real_huge.EINVAL, "bad plan")

    with pytest.raises(real_huge.HugeError):
        _batch_tuples(_Broken(), [(3, inputs.QUERIES["triangle"][1], [0, 1, 2])] * 2)


def test_good_order_starts_at_vertex_0_and_binds_the_best_connected_vertex_next():
    rng = np.random.default_rng(5)
    for name in ["k4", "c4", "house", "tailed_diamond_a", "path5", "c6"]:
        k, e = inputs.QUERIES[name]
        es = {frozenset(x) for x in map(tuple, e)}
        for _ in range(10):
            o = learned.good_order(k, e, rng)
            assert o[0] == 0 and sorted(o) == list(range(k))
            for j in range(1, k):
                def bound_nbrs(v):
                    return sum(frozenset((v, u)) in es for u in o[:j])

                assert bound_nbrs(o[j]) >= 1  # a connected prefix
                assert all(bound_nbrs(v) <= bound_nbrs(o[j]) for v in o[j:])
