"""Workload runs beyond the headline benchmark (each prints one JSON object).

  python -m paper_2103_14294_b300.experiments batch    # 256 random queries, R-MAT 22: one
                                                       # persistent launch vs 256 launches
  python -m paper_2103_14294_b300.experiments chunglu  # 5-vertex queries on Chung-Lu 4M/35M:
                                                       # COUNT, and LIST into a 4 GB device ring
  python -m paper_2103_14294_b300.experiments learned  # learned vs plain plans (see learned.py)
  python -m paper_2103_14294_b300.experiments motifs   # motif census of sizes 3-5, R-MAT 16:
                                                       # one batched launch per size vs one
                                                       # launch per pattern

Inputs are the seeded synthetic workloads of `inputs`. Parity of these workloads with the CPU
oracle (sampled roots, hubs included) is checked in tests/test_gpu_workloads.py; the runs here
check only what holds at any size (identical counts across forms, listed rows = count, sampled
listed rows are matches).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import huge


def _sync():
    import torch

    torch.cuda.synchronize()


def _order(k, edges, po):
    """A connected matching order that starts at a minimal element of the partial order and
    prefers vertices with more bound neighbours, then vertices bounded from below."""
    lt = set(po)
    adj = {v: set() for v in range(k)}
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    root = min(range(k), key=lambda v: (sum((u, v) in lt for u in range(k)), v))
    order = [root]
    while len(order) < k:
        best = max((v for v in range(k) if v not in order and adj[v] & set(order)),
                   key=lambda v: (2 * len(adj[v] & set(order)) + any((u, v) in lt for u in order), -v))
        order.append(best)
    return order


def _auto_po(G, k, edges):
    """The library's automatic symmetry-breaking partial order (read from a plan built with a
    given order, so no cardinality estimation runs)."""
    adj = {v: set() for v in range(k)}
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    order, seen = [0], {0}
    while len(order) < k:
        v = min(w for u in order for w in adj[u] if w not in seen)
        order.append(v)
        seen.add(v)
    p = huge.Plan(G, k, edges, order=order)
    po = [tuple(x) for x in p.describe()["po"]]
    p.free()
    return po


def _stratified(n, s, seed):
    rng = np.random.default_rng(seed)
    r = (np.arange(s) * (n / s) + rng.uniform(0, n / s, s)).astype(np.int64)
    return np.minimum(r, n - 1).astype(np.uint32)


def batch(scale=22, nq=256, work_limit=1e8, budget_ms=3000.0, mem_bound=16 << 30, seed0=40000,
          select_budget_s=240.0):
    """256 seeded random connected queries (3-6 vertices, random spanning tree + each other
    pair with probability 1/2, automatic partial orders) over R-MAT `scale`, each with a
    connected matching order. A query whose work estimated from 64 stratified roots (EXTEND
    applications x n / 64) exceeds work_limit is replaced by the next seed, so the whole run
    fits in minutes (selection stops after select_budget_s with the queries found so far).
    Compares the sequential launches with one batched launch (autotuned)."""
    import inputs

    t0 = time.time()
    g = inputs.rmat(scale, 16, 4)
    G = huge.Graph(g.offsets, g.adj, flags=huge.RELABEL_BY_DEGREE | huge.TRUST_SORTED)
    t_load = time.time() - t0
    roots = _stratified(g.n, 64, 1)
    plans, queries, skipped = [], [], 0
    s = seed0
    t0 = time.time()
    while len(plans) < nq and time.time() - t0 < select_budget_s:
        k = 3 + (s % 4)
        _, e = inputs.random_query(k, s)
        s += 1
        po = _auto_po(G, k, e)
        p = huge.Plan(G, k, e, order=_order(k, e, po))  # an upward connected order
        try:
            _, st = huge.enumerate(p, roots=roots, stats=True, time_limit_ms=200, mem_bound=mem_bound)
            work = st["intersections"] * g.n / len(roots)
        except huge.HugeError:
            work = float("inf")
        if work > work_limit:
            skipped += 1
            p.free()
            continue
        plans.append(p)
        queries.append((k, e))
    t_plan = time.time() - t0
    _sync()
    t0 = time.perf_counter()
    seq = [huge.enumerate(p, mem_bound=mem_bound, time_limit_ms=60000) for p in plans]
    _sync()
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    cap, chunk = huge.autotune(plans, mem_bound=mem_bound, budget_ms=budget_ms)
    t_tune = time.perf_counter() - t0
    _sync()
    t0 = time.perf_counter()
    bat, st = huge.enumerate_batch(plans, mem_bound=mem_bound, stats=True)
    _sync()
    t_bat = time.perf_counter() - t0
    t0 = time.perf_counter()
    bat2 = huge.enumerate_batch(plans, mem_bound=mem_bound)
    _sync()
    t_bat2 = time.perf_counter() - t0
    return {"workload": f"rmat{scale}-ef16-s4, {len(plans)} random connected queries (3-6 vertices)",
            "n": g.n, "m": g.m, "load_s": t_load, "select_s": t_plan, "skipped_over_limit": skipped,
            "sequential_s": t_seq, "batched_s": t_bat, "batched_s_second_run": t_bat2,
            "speedup": t_seq / t_bat2, "autotune_s": t_tune, "tuned_level_cap": cap, "tuned_chunk": chunk,
            "counts_identical": bool(list(seq) == list(bat) == list(bat2)),
            "total_matches": int(sum(seq)), "batched_device_ms": st["device_ms"],
            "query_sizes": [k for k, _ in queries]}


def motif_census(scale=16, ks=(3, 4, 5), mem_bound=8 << 30):
    """Motif census (Sec. 6, graph pattern mining) on R-MAT `scale` (edge factor 16): for each
    size, all connected patterns as one batched launch against one launch per pattern; the
    non-induced counts must be identical, the induced ones follow exactly."""
    import inputs

    from . import motifs

    g = inputs.rmat(scale, 16, 60 + scale)
    G = huge.Graph(g.offsets, g.adj)
    out = {"workload": f"rmat{scale}-ef16-s{60 + scale}", "n": g.n, "m": g.m, "sizes": {}}
    for k in ks:
        _sync()
        t0 = time.perf_counter()
        rows = motifs.census(G, k, mem_bound=mem_bound)
        _sync()
        t_bat = time.perf_counter() - t0
        t0 = time.perf_counter()
        seq = []
        for p in motifs.patterns(k):
            plan = huge.Plan(G, k, list(p), order=motifs._order(k, p))
            seq.append(huge.enumerate(plan, mem_bound=mem_bound))
            plan.free()
        _sync()
        t_seq = time.perf_counter() - t0
        out["sizes"][k] = {"patterns": len(rows), "batched_s": t_bat, "sequential_s": t_seq,
                           "counts_identical": [r[1] for r in rows] == seq,
                           "induced": [r[2] for r in rows], "noninduced": [r[1] for r in rows]}
    return out


def chunglu(ring_gb=4.0, mem_bound=32 << 30, verify_rows=4000, limit_ms=120000, list_hubs_excluded=5000,
            sample_stride=4096):
    """5-clique, house and tailed diamond on the Chung-Lu graph (4,194,304 vertices, 35M
    edges, exponent 2.1, max weight 15,000).
      * 5-clique: exact COUNT over all roots; LIST into a device ring of ring_gb GB, drained to
        the host, over every root but the `list_hubs_excluded` largest (the listed rows of the
        full range would be ~0.9 TB); the listed rows must equal the COUNT of that range and a
        sample of every drain is checked: mapped back to the original ids, rows are matches
        (query edges present, distinct vertices) obeying the partial order on relabelled ids.
      * house, tailed diamond: their counts are of order 1e14-1e15 on this graph, beyond a
        minutes budget; COUNT and LIST on a stratified 1/sample_stride root sample."""
    import torch

    import inputs

    t0 = time.time()
    g = inputs.chung_lu(4 * 1024 * 1024, 35_000_000, 3)
    t_gen = time.time() - t0
    G = huge.Graph(g.offsets, g.adj, flags=huge.RELABEL_BY_DEGREE | huge.TRUST_SORTED)
    old_of_new = np.argsort(G.new_ids()).astype(np.int64)
    deg = np.diff(g.offsets).astype(np.int64)
    keys = np.repeat(np.arange(g.n, dtype=np.int64), deg) * (1 << 32) + g.adj.astype(np.int64)  # sorted
    out = {"workload": "chunglu-4194304-35000000-s3", "n": g.n, "m": g.m,
           "max_degree": int(deg.max()), "gen_s": t_gen, "queries": {}}
    k_ring = 5
    ring_rows = int(ring_gb * (1 << 30)) // (4 * k_ring)
    ring = torch.empty((ring_rows, k_ring), dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(3)

    def checker(k, e, po, drained):
        def drain(ptr, nrows):
            drained["rows"] += nrows
            drained["chunks"] += 1
            take = min(verify_rows, nrows)
            idx = torch.from_numpy(np.sort(rng.choice(nrows, take, replace=False))).cuda()
            rows = ring[:nrows].index_select(0, idx).cpu().numpy().astype(np.int64)
            ok = np.ones(take, dtype=bool)
            for a, b in po:
                ok &= rows[:, a] < rows[:, b]
            orig = old_of_new[rows]
            for a, b in e:
                q = orig[:, a] * (1 << 32) + orig[:, b]
                pos = np.minimum(np.searchsorted(keys, q), len(keys) - 1)
                ok &= keys[pos] == q
            srt = np.sort(rows, axis=1)
            ok &= np.all(srt[:, 1:] != srt[:, :-1], axis=1)
            drained["checked"] += take
            drained["bad"] += int((~ok).sum())
        return drain

    for name in ("k5", "house", "tailed_diamond_a"):
        try:
            out["queries"][name] = _chunglu_query(G, g, name, ring, ring_rows, checker, mem_bound, limit_ms,
                                                  list_hubs_excluded, sample_stride)
        except huge.HugeError as err:
            out["queries"][name] = {"error": str(err)[:300]}
    return out


def _chunglu_query(G, g, name, ring, ring_rows, checker, mem_bound, limit_ms, list_hubs_excluded, sample_stride):
    import inputs

    k, e = inputs.QUERIES[name]
    po = _auto_po(G, k, e)
    p = huge.Plan(G, k, e, order=_order(k, e, po))
    d = p.describe()
    rec = {"order": d["chain"]["order"], "po": po}
    if name == "k5":
        _sync()
        t0 = time.perf_counter()
        c, st = huge.enumerate(p, mem_bound=mem_bound, stats=True, time_limit_ms=limit_ms)
        rec.update({"count": c, "count_s": time.perf_counter() - t0, "device_ms": st["device_ms"],
                    "matches_per_s": c / (st["device_ms"] / 1e3), "intersections": st["intersections"],
                    "level_rows": st["level_rows"]})
        rr = (0, g.n - list_hubs_excluded)
        c_rr = huge.enumerate(p, mem_bound=mem_bound, root_range=rr, time_limit_ms=limit_ms)
        drained = {"rows": 0, "chunks": 0, "checked": 0, "bad": 0}
        _sync()
        t0 = time.perf_counter()
        cl = huge.enumerate(p, mode=huge.LIST, sink=ring, mem_bound=mem_bound, root_range=rr,
                            drain=checker(k, e, po, drained), time_limit_ms=limit_ms)
        _sync()
        rec.update({"list_root_range": list(rr), "count_in_range": c_rr, "list_count": cl,
                    "list_s": time.perf_counter() - t0, "ring_rows": ring_rows, **{f"drain_{x}": v for x, v in
                                                                                      drained.items()},
                    "list_equals_count": bool(cl == c_rr == drained["rows"])})
    else:
        roots = _stratified(g.n, g.n // sample_stride, 9)
        _sync()
        t0 = time.perf_counter()
        try:
            c, st = huge.enumerate(p, mem_bound=mem_bound, stats=True, roots=roots, time_limit_ms=limit_ms)
            rec.update({"sample_roots": int(len(roots)), "sample_count": c,
                        "count_s": time.perf_counter() - t0, "device_ms": st["device_ms"],
                        "matches_per_s": c / (st["device_ms"] / 1e3), "extrapolated_count": c * sample_stride,
                        "level_rows": st["level_rows"]})
        except huge.HugeError as err:
            rec["sample_count_error"] = str(err)[:300]
        # LIST on roots outside the dense core (the core's rows alone would be terabytes)
        lroots = _stratified(g.n - 20000, 2048, 11)
        cl_count = huge.enumerate(p, mem_bound=mem_bound, roots=lroots, time_limit_ms=limit_ms)
        rec.update({"list_roots": "2048 stratified roots below the 20000 largest ids", "list_root_count": cl_count})
        if cl_count <= 4 * ring_rows:
            drained = {"rows": 0, "chunks": 0, "checked": 0, "bad": 0}
            t0 = time.perf_counter()
            cl = huge.enumerate(p, mode=huge.LIST, sink=ring, mem_bound=mem_bound, roots=lroots,
                                drain=checker(k, e, po, drained), time_limit_ms=limit_ms)
            rec.update({"list_count": cl, "list_s": time.perf_counter() - t0,
                        **{f"drain_{x}": v for x, v in drained.items()},
                        "list_equals_count": bool(cl == cl_count == drained["rows"])})
    p.free()
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["batch", "chunglu", "learned", "motifs"])
    ap.add_argument("--scale", type=int, default=None, help="R-MAT scale (batch: 22, motifs: 16)")
    ap.add_argument("--nq", type=int, default=256)
    ap.add_argument("--select-budget-s", type=float, default=240.0)
    ap.add_argument("--limit-ms", type=int, default=120000)
    args, rest = ap.parse_known_args()
    if args.what == "batch":
        print(json.dumps(batch(scale=args.scale or 22, nq=args.nq, select_budget_s=args.select_budget_s)))
    elif args.what == "chunglu":
        print(json.dumps(chunglu(limit_ms=args.limit_ms)))
    elif args.what == "motifs":
        print(json.dumps(motif_census(scale=args.scale or 16)))
    else:
        from . import learned

        sys.argv = [sys.argv[0]] + rest
        learned.main()
    return 0


if __name__ == "__main__":
    sys.exit(main())
