"""The multi-rank path on CPU (gloo, world size 2): root shards cover every root once and their
counts add up to the whole count; the benchmark's whole-job aggregation takes the slowest
rank's time and the sum of the ranks' matches."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import inputs
    import oracle
    from paper_2103_14294_b300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = inputs.rmat(9, 8, 11)
        gr, _ = oracle.relabel_by_degree(g)
        r0, r1 = shard.shard_of(gr.offsets, rank, world)
        res = {}
        for name in ("triangle", "c4", "tailed_diamond_a"):
            k, e = inputs.QUERIES[name]
            po = oracle.symmetry_breaking_order(k, e)
            order = oracle.connected_order(k, e)
            roots = np.arange(r0, r1, dtype=np.uint32)
            local = int(oracle.count_roots(gr, k, e, roots, po, order, threads=1).sum())
            t = torch.tensor([local], dtype=torch.int64)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            res[name] = (int(t[0]), int(oracle.count(gr, k, e, po)))
        t_job, m_job = bench.job_totals(1.0 + rank, 10 * (rank + 1), torch.device("cpu"), world)
        res["job"] = (t_job, m_job)
        res["shard"] = (r0, r1)
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_roots_and_aggregate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    r0, r1 = out[0], out[1]
    assert r0["shard"][0] == 0 and r0["shard"][1] == r1["shard"][0]
    for name in ("triangle", "c4", "tailed_diamond_a"):
        got, want = r0[name]
        assert got == want and r1[name] == (got, want), name
    assert r0["job"] == (2.0, 30.0) and r1["job"] == (2.0, 30.0)


def test_shard_bounds_cover_and_balance():
    from paper_2103_14294_b300 import shard

    off = np.concatenate([[0], np.cumsum(np.r_[np.full(90, 1), np.full(10, 100)])])
    for world in (1, 2, 3, 7):
        b = shard.shard_bounds(off, world)
        assert b[0][0] == 0 and b[-1][1] == 100
        assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
    b = shard.shard_bounds(off, 2)
    w = 1 + np.diff(off)
    assert abs(int(w[b[0][0]:b[0][1]].sum()) - int(w[b[1][0]:b[1][1]].sum())) <= int(w.max())
    assert shard.shard_bounds(np.zeros(1, np.int64), 3) == [(0, 0)] * 3
    with pytest.raises(ValueError):
        shard.shard_of(off, 2, 2)


def test_relabelled_offsets_match_the_relabelled_graph():
    """Root ranges are cut on the degree sequence in the library's ids: the sorted degrees,
    which is exactly the CSR offsets of the graph relabelled by (degree, id)."""
    sys.path.insert(0, ROOT)
    import inputs
    import oracle
    from paper_2103_14294_b300 import shard

    for g in (inputs.rmat(10, 8, 3), inputs.er(500, 3000, 4)):
        gr, _ = oracle.relabel_by_degree(g)
        assert np.array_equal(shard.relabelled_offsets(g), gr.offsets.astype(np.int64))
