"""Workload runs beyond the headline benchmark (each prints one JSON object).

  python -m paper_2103_14294_b300.experiments batch    # 256 random queries, R-MAT 22: one
                                                       # persistent launch vs 256 launches
  python -m paper_2103_14294_b300.experiments chunglu  # 5-vertex queries on Chung-Lu 4M/35M:
                                                       # COUNT, and LIST into a 4 GB device ring
  python -m paper_2103_14294_b300.experiments learned  # learned vs plain plans (see learned.py)
  python -m paper_2103_14294_b300.experiments outofcore  # R-MAT 20 K4 / C4 with 100..0% of the
                                                       # adjacency in HBM, the rest in host memory
  python -m paper_2103_14294_b300.experiments motifs   # motif census of sizes 3-5, R-MAT 12:
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


def batch(scale=22, nq=256, target_ms=4.0, mem_bound=16 << 30, seed0=40000, probe_roots=64,
          probe_limit_ms=2000, run_limit_ms=20000):
    """256 seeded random connected queries (3-6 vertices, random spanning tree + each other
    pair with probability 1/2, automatic partial orders, a connected upward matching order)
    over R-MAT `scale`. Every query keeps its place; its work is bounded by a root sample
    instead: a probe over `probe_roots` stratified roots estimates the device time per root,
    and the query then runs on a stratified sample sized for about `target_ms` of device time
    (at least one root). Compares 256 plain launches (one per query, each on its own roots)
    with ONE batched persistent launch over all (query, root) tasks, heaviest first; counts
    must be identical per query."""
    import inputs

    t0 = time.time()
    g = inputs.rmat(scale, 16, 4)
    G = huge.Graph(g.offsets, g.adj, flags=huge.RELABEL_BY_DEGREE | huge.TRUST_SORTED)
    t_load = time.time() - t0
    plans, queries, roots, bands = [], [], [], []
    t0 = time.time()
    for i in range(nq):
        k = 3 + (i % 4)
        _, e = inputs.random_query(k, seed0 + i)
        po = _auto_po(G, k, e)
        p = huge.Plan(G, k, e, order=_order(k, e, po))
        # probe the whole id range, else the lower half (the low-degree roots), else one root of
        # the lowest degree; the sample then covers the band the probe finished on
        chosen = None
        for hi in (g.n, g.n // 2):
            probe = _stratified(hi, probe_roots, 1)
            try:
                _, st = huge.enumerate(p, roots=probe, stats=True, time_limit_ms=probe_limit_ms, mem_bound=mem_bound)
            except huge.HugeError:
                continue
            per_root = max(st["device_ms"], 1e-3) / len(probe)
            chosen = (hi, int(min(hi, max(1, target_ms / per_root))))
            break
        if chosen is None:
            chosen = (1, 1)
        plans.append(p)
        queries.append((k, e))
        roots.append(_stratified(chosen[0], chosen[1], 1000 + i))
        bands.append(chosen[0])
    t_select = time.time() - t0
    _sync()
    # plain: one launch per query on its roots; a query whose plain launch exceeds the run
    # limit is dropped from both forms (reported)
    t0 = time.perf_counter()
    seq, seq_dev, keep = [], 0.0, []
    for i, (p, r) in enumerate(zip(plans, roots)):
        try:
            c, st = huge.enumerate(p, roots=r, mem_bound=mem_bound, time_limit_ms=run_limit_ms, stats=True)
        except huge.HugeError:
            continue
        seq.append(c)
        seq_dev += st["device_ms"]
        keep.append(i)
    _sync()
    t_seq = time.perf_counter() - t0
    dropped = [i for i in range(len(plans)) if i not in keep]
    if dropped:  # time the plain form again over the kept queries only
        _sync()
        t0 = time.perf_counter()
        for i in keep:
            huge.enumerate(plans[i], roots=roots[i], mem_bound=mem_bound, time_limit_ms=run_limit_ms)
        _sync()
        t_seq = time.perf_counter() - t0
    plans = [plans[i] for i in keep]
    roots = [roots[i] for i in keep]
    queries = [queries[i] for i in keep]
    runs = []
    for _ in range(2):
        _sync()
        t0 = time.perf_counter()
        bat, st = huge.enumerate_batch(plans, roots=roots, mem_bound=mem_bound, stats=True,
                                       time_limit_ms=run_limit_ms)
        _sync()
        runs.append((time.perf_counter() - t0, st["device_ms"], list(bat)))
    return {"workload": f"rmat{scale}-ef16-s4, {len(plans)} random connected queries (3-6 vertices), "
                        f"each on a stratified root sample sized for ~{target_ms} ms of device time",
            "n": g.n, "m": g.m, "load_s": t_load, "select_s": t_select,
            "query_sizes": {str(k): sum(1 for q in queries if q[0] == k) for k in range(3, 7)},
            "dropped_over_run_limit": dropped,
            "root_band": {"whole": sum(1 for b in bands if b == g.n), "lower_half": sum(1 for b in bands if b == g.n // 2),
                          "one_root": sum(1 for b in bands if b == 1)},
            "roots_per_query": {"min": int(min(map(len, roots))), "median": int(np.median(list(map(len, roots)))),
                                "max": int(max(map(len, roots))), "total": int(sum(map(len, roots)))},
            "plain_launches": len(plans), "plain_s": t_seq, "plain_device_ms": seq_dev,
            "batched_s": [r[0] for r in runs], "batched_device_ms": [r[1] for r in runs],
            "speedup_end_to_end": t_seq / min(r[0] for r in runs),
            "counts_identical": bool(all(r[2] == list(seq) for r in runs)),
            "total_matches": int(sum(seq))}


def motif_census(scale=12, ks=(3, 4, 5), mem_bound=8 << 30):
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
            sample_stride=256, full_budget_s=150.0):
    """5-clique, house and tailed diamond on the Chung-Lu graph (4,194,304 vertices, 35M
    edges, exponent 2.1, max weight 15,000).
      * 5-clique: exact COUNT over all roots; LIST into a device ring of ring_gb GB, drained to
        the host, over every root but the `list_hubs_excluded` largest (the listed rows of the
        full range would be ~0.9 TB); the listed rows must equal the COUNT of that range and a
        sample of every drain is checked: mapped back to the original ids, rows are matches
        (query edges present, distinct vertices) obeying the partial order on relabelled ids.
      * house, tailed diamond: COUNT on a stratified 1/sample_stride root sample; when the
        sample's device time extrapolates to under full_budget_s, COUNT over every root too.
        LIST of 2048 stratified roots outside the dense core.
    SM clocks are sampled during the whole run; peak_bytes is the intermediate-result memory
    the launch held (per-warp level buffers and the donation pool) against mem_bound."""
    import torch

    import inputs

    from .clocks import ClockSampler

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

    with ClockSampler(torch.cuda.current_device()) as clk:
        for name in ("k5", "house", "tailed_diamond_a"):
            try:
                out["queries"][name] = _chunglu_query(G, g, name, ring, ring_rows, checker, mem_bound, limit_ms,
                                                      list_hubs_excluded, sample_stride, full_budget_s)
            except huge.HugeError as err:
                out["queries"][name] = {"error": str(err)[:300]}
    out["clocks"] = clk.summary()
    out["mem_bound_bytes"] = mem_bound
    return out


def _chunglu_query(G, g, name, ring, ring_rows, checker, mem_bound, limit_ms, list_hubs_excluded, sample_stride,
                   full_budget_s):
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
                    "level_rows": st["level_rows"], "peak_bytes": st["peak_bytes"], "level_cap": st["level_cap"]})
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
                        "level_rows": st["level_rows"], "peak_bytes": st["peak_bytes"]})
            if st["device_ms"] * sample_stride / 1e3 < full_budget_s:
                _sync()
                t0 = time.perf_counter()
                cf, stf = huge.enumerate(p, mem_bound=mem_bound, stats=True, time_limit_ms=int(2e3 * full_budget_s))
                rec.update({"count": cf, "count_full_s": time.perf_counter() - t0, "device_ms_full": stf["device_ms"],
                            "matches_per_s_full": cf / (stf["device_ms"] / 1e3), "peak_bytes_full": stf["peak_bytes"],
                            "level_rows_full": stf["level_rows"]})
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


def er_triangles(reps=5):
    """The K3 workload (ER n=2000, m=20000, partial order v0<v1<v2): device time of the exact
    count, best of `reps`, for every matching order."""
    import itertools

    import inputs

    g = inputs.workload_graph("er2000")
    G = huge.Graph(g.offsets, g.adj)
    k, e = inputs.QUERIES["triangle"]
    out = {"workload": "er2000 triangles", "n": g.n, "m": g.m, "orders": {}}
    for o in itertools.permutations(range(3)):
        p = huge.Plan(G, k, e, order=list(o), po=[(0, 1), (1, 2), (0, 2)])
        best, c = None, None
        for _ in range(reps):
            c, st = huge.enumerate(p, stats=True)
            best = st["device_ms"] if best is None else min(best, st["device_ms"])
        out["orders"]["".join(map(str, o))] = {"count": c, "device_ms": best}
    return out


def outofcore(scale=20, fractions=(1.0, 0.5, 0.25, 0.1, 0.0), mem_bound=8 << 30):
    """The benchmark's 4-clique and 4-cycle counts on R-MAT `scale` with only a fraction of
    the adjacency array in HBM (the lists of the highest-degree vertices) and the rest read from
    host memory: device time per query and identical counts at every budget."""
    import inputs

    g = inputs.rmat(scale, 16, 2)
    G = huge.Graph(g.offsets, g.adj)
    adj_bytes = ((g.nnz + 3) // 4 * 4 + 4) * 4
    orders = {"k4": [0, 3, 2, 1], "c4": [0, 3, 1, 2]}
    plans = {n: huge.Plan(G, *inputs.QUERIES[n], order=o) for n, o in orders.items()}
    out = {"workload": f"rmat{scale}-ef16-s2", "adj_bytes": adj_bytes, "hub_bitmaps": G.hub_info(), "runs": []}
    for f in fractions:
        resident = G.set_residency(int(adj_bytes * f) if f < 1 else 1 << 62)
        row = {"fraction": f, "resident_bytes": resident}
        for n, p in plans.items():
            c, st = huge.enumerate(p, mem_bound=mem_bound, stats=True)
            c2, st2 = huge.enumerate(p, mem_bound=mem_bound, stats=True)
            row[n] = {"count": c, "device_ms": min(st["device_ms"], st2["device_ms"]), "repeat_equal": c == c2}
        out["runs"].append(row)
    out["counts_identical"] = all(r[n]["count"] == out["runs"][0][n]["count"] for r in out["runs"] for n in orders)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["batch", "chunglu", "learned", "motifs", "outofcore", "er2000"])
    ap.add_argument("--scale", type=int, default=None, help="R-MAT scale (batch: 22, motifs: 16)")
    ap.add_argument("--nq", type=int, default=256)
    ap.add_argument("--target-ms", type=float, default=4.0)
    ap.add_argument("--limit-ms", type=int, default=120000)
    args, rest = ap.parse_known_args()
    if args.what == "batch":
        print(json.dumps(batch(scale=args.scale or 22, nq=args.nq, target_ms=args.target_ms)))
    elif args.what == "chunglu":
        print(json.dumps(chunglu(limit_ms=args.limit_ms)))
    elif args.what == "er2000":
        print(json.dumps(er_triangles()))
    elif args.what == "outofcore":
        print(json.dumps(outofcore(scale=args.scale or 20)))
    elif args.what == "motifs":
        print(json.dumps(motif_census(scale=args.scale or 12)))
    else:
        from . import learned

        sys.argv = [sys.argv[0]] + rest
        learned.main()
    return 0


if __name__ == "__main__":
    sys.exit(main())
