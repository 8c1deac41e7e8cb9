"""The enumerator's per-warp scheduling policy, modelled on the host next to Alg. 5.

The persistent kernel departs from Alg. 5 (Sec. 5.2) in granularity. Each level holds at most
`cap` rows. A warp extends one batch of at most 32 input rows, stopping as soon as the next
level is full, and remembers where it stopped: which row, and how far into that row's
candidate list. It then returns to the deepest level that has input. This model replays that
policy with the EXTEND semantics of ``oracle.scheduler.extend_ops``. It checks three claims:

* the count is the oracle's, whatever the capacity and batch size;
* no level ever holds more than `cap` rows. Alg. 5 can overshoot by one batch's output, up
  to D_G batches by Lemma 5.1; here the bound does not depend on D_G;
* the policy always makes progress: every step moves at least one row or candidate.
"""
import numpy as np
import pytest

import inputs
import oracle
from oracle import scheduler


def _candidates(adj, k, edges, order, po):
    """cand(row) -> the sorted candidates of the next position, from the same EXTEND rules as
    oracle.scheduler.extend_ops (one input row at a time)."""
    _, ops = scheduler.extend_ops(adj, k, edges, order, po, batch_rows=1 << 30)
    scan, extends = ops[0], ops[1:-1]

    def cand(level, row):
        if level == 0:  # the edge scan from a root
            out = scan(row[0])
            return [r[1] for r in (out[0] if out else [])]
        out = extends[level - 1]([row])
        return [r[-1] for r in (out[0] if out else [])]

    return cand


def run_deepest_first(adj, k, edges, order, po, cap, batch):
    """The warp's policy. Levels 0..k-1 hold rows of 1..k vertices (level 0: the roots, a
    source consumed in order). Returns (count, the most rows any level held, steps)."""
    cand = _candidates(adj, k, edges, order, po)
    levels = [[] for _ in range(k)]  # pending rows per level (level k-1: complete matches)
    cursor = [None] * k  # (row, candidates, next index) of a row stopped mid-list
    roots = list(range(len(adj)))
    count, peak, steps = 0, [0] * k, 0
    while True:
        # the deepest level with work: a stopped row or pending rows; else the next roots
        lvl = next((l for l in range(k - 2, 0, -1) if cursor[l] or levels[l]), None)
        if lvl is None:
            if cursor[0] is None and not roots:
                break
            lvl = 0
        steps += 1
        moved = 0
        taken = 0
        while taken < batch:
            if cursor[lvl] is None:
                if lvl == 0:
                    if not roots:
                        break
                    row = (roots.pop(0),)
                else:
                    if not levels[lvl]:
                        break
                    row = levels[lvl].pop(0)
                cursor[lvl] = (row, cand(lvl, row), 0)
                taken += 1
            row, cs, i = cursor[lvl]
            if lvl + 1 == k - 1:  # the last operator: count, nothing is stored
                count += len(cs) - i
                moved += len(cs) - i
                cursor[lvl] = None
                continue
            room = cap - len(levels[lvl + 1])
            take = min(room, len(cs) - i)
            levels[lvl + 1].extend(row + (u,) for u in cs[i:i + take])
            peak[lvl + 1] = max(peak[lvl + 1], len(levels[lvl + 1]))
            moved += take
            if i + take < len(cs):  # the next level is full: stop inside this row
                cursor[lvl] = (row, cs, i + take)
                break
            cursor[lvl] = None
        assert moved > 0 or taken > 0, "a scheduling step made no progress"
    return count, max(peak), steps


@pytest.mark.parametrize("name", ["triangle", "k4", "c4", "house", "tailed_diamond_a", "k5"])
def test_deepest_first_policy_counts_and_strict_bound(name):
    g = oracle.relabel_by_degree(inputs.gnp(40, 1, 4, 17))[0]
    off = np.asarray(g.offsets, dtype=np.int64)
    adj = [set(map(int, g.adj[off[u]:off[u + 1]])) for u in range(g.n)]
    k, e = inputs.QUERIES[name]
    po = oracle.symmetry_breaking_order(k, e)
    order = oracle.connected_order(k, e)
    want = oracle.count(g, k, e, po)
    for cap in (1, 2, 7, 64):
        for batch in (1, 32):
            got, peak, _ = run_deepest_first(adj, k, e, order, po, cap, batch)
            assert got == want, (name, cap, batch)
            assert peak <= cap, (name, cap, batch, peak)


def test_alg5_overshoots_where_the_warp_policy_does_not():
    """On a hub, one input batch of Alg. 5 can produce far more than a queue holds; the warp
    policy stops inside the hub's list instead. Same count either way."""
    from inputs import Graph

    n = 60
    hub_edges = [(0, v) for v in range(1, n)]  # a star: the hub has degree n - 1
    nb = [[] for _ in range(n)]
    for a, b in hub_edges:
        nb[a].append(b)
        nb[b].append(a)
    off = np.concatenate([[0], np.cumsum([len(x) for x in nb])]).astype(np.uint64)
    g = Graph(off, np.asarray([v for x in nb for v in sorted(x)], dtype=np.uint32), "star60")
    adj = [set(x) for x in nb]
    k, e = 3, [(0, 1), (0, 2)]  # a wedge centred on the first vertex
    po = oracle.symmetry_breaking_order(k, e)
    order = [0, 1, 2]
    want = oracle.count(g, k, e, po)
    source, ops = scheduler.extend_ops(adj, k, e, order, po, batch_rows=4)
    res = scheduler.run(source, ops, cap=2)
    assert sum(res["sink"]) == want
    assert max(res["peak"][:-1]) > 2  # Alg. 5: the hub's edge scan overfills its queue
    got, peak, _ = run_deepest_first(adj, k, e, order, po, cap=8, batch=4)
    assert got == want and peak <= 8
