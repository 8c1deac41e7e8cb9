"""Learned cardinality estimator around the library: training tuples logged by the exact
enumerator, GPU training of the tensor-core MLP, and plain-vs-learned plan comparisons.

A training tuple is (features of a sub-query q', log(1 + |R(q')|)). Every exact enumeration of
an EXTEND chain logs |R| of each prefix of its matching order (the per-level row counts of
huge_enumerate_ex), so one run yields one tuple per prefix of three or more vertices; the
features are the ones the planner uses (huge_plan_features), so training and planning see the
same inputs. The network then replaces the sampling estimator inside Alg. 1 (HUGE_PLAN_LEARNED).

  python -m paper_2103_14294_b300.learned --tuples 50000 --out model.npz --eval-scale 23
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from . import huge


def random_connected_order(k, edges, rng):
    adj = {v: set() for v in range(k)}
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    order = [int(rng.integers(k))]
    while len(order) < k:
        cand = sorted({w for v in order for w in adj[v]} - set(order))
        order.append(int(cand[rng.integers(len(cand))]))
    return order


def log_tuples(G, k, edges, order, time_limit_ms=2000, mem_bound=4 << 30):
    """Exact per-prefix counts of one EXTEND chain -> [(mask, log1p(count))] for prefixes >= 3,
    or [] when the run exceeds its time limit or overflows."""
    p = huge.Plan(G, k, edges, order=order)
    try:
        _, st = huge.enumerate(p, stats=True, time_limit_ms=time_limit_ms, mem_bound=mem_bound)
    except huge.HugeError as e:
        if e.code in (huge.ETIMEOUT, huge.EOVERFLOW):
            return []
        raise
    out = []
    rows = st["level_rows"]
    for i in range(2, k):
        mask = sum(1 << v for v in order[: i + 1])
        out.append((mask, math.log1p(rows[i])))
    return out


def _batch_tuples(G, items, time_limit_ms, mem_bound, out):
    """Exact per-prefix counts of many (k, edges, order) chains in one batched launch; a batch
    that reaches the time limit is split in halves (a single chain that does is dropped)."""
    if not items:
        return
    plans = [huge.Plan(G, k, e, order=o) for k, e, o in items]
    lr = np.zeros((len(plans), 16), dtype=np.int64)
    try:
        counts = huge.enumerate_batch(plans, level_rows=lr, time_limit_ms=time_limit_ms, mem_bound=mem_bound)
    except huge.HugeError as err:
        for p in plans:
            p.free()
        if err.code not in (huge.ETIMEOUT, huge.EOVERFLOW) or len(items) == 1:
            if err.code in (huge.ETIMEOUT, huge.EOVERFLOW):
                return
            raise
        h = len(items) // 2
        _batch_tuples(G, items[:h], time_limit_ms, mem_bound, out)
        _batch_tuples(G, items[h:], time_limit_ms, mem_bound, out)
        return
    for (k, e, o), p, row, c in zip(items, plans, lr, counts):
        p.free()
        for i in range(2, k):  # prefix of i + 1 vertices: rows at level i, the count at the end
            y = int(c) if i == k - 1 else int(row[i])
            out.append((k, e, sum(1 << v for v in o[: i + 1]), math.log1p(y)))


def good_order(k, edges, rng):
    """A connected matching order that chains upward: it starts at vertex 0, which the automatic
    partial order never places above another vertex (symmetry breaking constrains the smallest
    vertex of a non-trivial orbit to lie below the rest of it), then prefers vertices with more
    bound neighbours (ties at random), so the exact run that logs the tuples rarely explodes."""
    adj = {v: set() for v in range(k)}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    order = [0]
    while len(order) < k:
        cand = [v for v in range(k) if v not in order and adj[v] & set(order)]
        best = max(len(adj[v] & set(order)) for v in cand)
        top = [v for v in cand if len(adj[v] & set(order)) == best]
        order.append(int(top[rng.integers(len(top))]))
    return order


def collect_batched(graphs, n_tuples, seed=0, batch=32, time_limit_ms=100, budget_s=300.0, verbose=False,
                    kmax=None, mem_bound=4 << 30, random_order_share=0.3):
    """As collect, with the exact runs of `batch` random (query, order) chains per graph issued as
    one batched launch (per-plan level rows), which makes tuples far cheaper to log. Most orders
    chain upward (good_order); a share are random connected orders, for sub-query variety."""
    import inputs

    rng = np.random.default_rng(seed)
    X, Y, meta = [], [], []
    t0 = time.time()
    qseed = seed * 1_000_003
    last = 0
    while len(Y) < n_tuples and time.time() - t0 < budget_s:
        for name, G in graphs:
            items = []
            for _ in range(batch):
                qseed += 1
                k = int(rng.integers(3, 1 + (kmax or {}).get(name, 6)))
                _, e = inputs.random_query(k, qseed)
                o = random_connected_order(k, e, rng) if rng.random() < random_order_share else good_order(k, e, rng)
                items.append((k, e, o))
            rows = []
            _batch_tuples(G, items, time_limit_ms, mem_bound, rows)
            for k, e, mask, y in rows:
                X.append(huge.plan_features(G, k, e, mask))
                Y.append(y)
                meta.append((name, k, mask))
            if len(Y) >= n_tuples or time.time() - t0 >= budget_s:
                break
        if verbose and len(Y) >= last + 5000:
            last = len(Y)
            print(f"  {len(Y)} tuples, {time.time() - t0:.0f}s", file=sys.stderr, flush=True)
    return np.asarray(X, np.float32), np.asarray(Y, np.float32), meta


def collect(graphs, n_tuples, seed=0, time_limit_ms=2000, budget_s=600.0, verbose=False, kmax=None):
    """Training set from exact runs of random connected queries (3-6 vertices, automatic partial
    orders, random connected matching orders) over the given graphs (list of (name, Graph)).
    kmax (dict name -> largest query size) keeps the queries on large graphs small; runs that
    exceed time_limit_ms are dropped."""
    import inputs

    rng = np.random.default_rng(seed)
    X, Y, meta = [], [], []
    t0 = time.time()
    qseed = seed * 1_000_003
    last = 0
    while len(Y) < n_tuples and time.time() - t0 < budget_s:
        for name, G in graphs:
            qseed += 1
            k = int(rng.integers(3, 1 + (kmax or {}).get(name, 6)))
            _, e = inputs.random_query(k, qseed)
            order = random_connected_order(k, e, rng)
            for mask, y in log_tuples(G, k, e, order, time_limit_ms):
                X.append(huge.plan_features(G, k, e, mask))
                Y.append(y)
                meta.append((name, k, mask))
        if verbose and len(Y) >= last + 2000:
            last = len(Y)
            print(f"  {len(Y)} tuples, {time.time() - t0:.0f}s", file=sys.stderr, flush=True)
    return np.asarray(X, np.float32), np.asarray(Y, np.float32), meta


def train(X, Y, seed=0, epochs=300, batch_rows=4096, lr=1e-3, holdout=0.1):
    """Trains a fresh MLP on the GPU; returns (model, train loss, holdout RMSE in log units)."""
    import torch

    rng = np.random.default_rng(seed)
    idx = rng.permutation(len(Y))
    nh = int(len(Y) * holdout)
    te, tr = idx[:nh], idx[nh:]
    mu = X[tr].mean(0)
    sd = X[tr].std(0) + 1e-3
    m = huge.MLP(seed)
    m.set_params(None, mu, sd)
    dx = torch.from_numpy(X[tr]).cuda()
    dy = torch.from_numpy(Y[tr]).cuda()
    loss = m.train(dx, dy, epochs=epochs, batch_rows=batch_rows, lr=lr)
    rmse = None
    if nh:
        out = torch.zeros(nh, dtype=torch.float32, device="cuda")
        m.forward(torch.from_numpy(X[te]).cuda(), out)
        rmse = float(np.sqrt(np.mean((out.cpu().numpy() - Y[te]) ** 2)))
    return m, loss, rmse


def save(model, path):
    p, mu, sd = model.get_params()
    np.savez(path, params=p, mu=mu, sd=sd)


def load_model(path, seed=0):
    d = np.load(path)
    m = huge.MLP(seed)
    m.set_params(d["params"], d["mu"], d["sd"])
    return m


def compare(G, queries, model, time_limit_ms=120000, mem_bound=16 << 30):
    """Plain optimiser (sampling estimator) vs learned estimator on each query: plan time,
    enumeration device time, the chosen plans' actual intermediate sizes, and the counts (which
    must be identical)."""
    res = []
    for k, e in queries:
        row = {"k": k, "edges": e}
        for tag, flags, mdl in (("plain", huge.PLAN_PLAIN, None), ("learned", huge.PLAN_LEARNED, model)):
            t0 = time.perf_counter()
            p = huge.Plan(G, k, e, flags=flags, model=mdl)
            t_plan = time.perf_counter() - t0
            t1 = time.perf_counter()
            try:
                c, st = huge.enumerate(p, stats=True, time_limit_ms=time_limit_ms, mem_bound=mem_bound)
            except huge.HugeError as err:
                c, st = None, {"error": str(err)}
            t_enum = time.perf_counter() - t1
            d = p.describe()
            row[tag] = {"plan_s": t_plan, "enum_s": t_enum, "e2e_s": t_plan + t_enum, "count": c,
                        "device_ms": st.get("device_ms"), "level_rows": st.get("level_rows"),
                        "op": d["op"], "order": d.get("chain", {}).get("order"), "est_cost": d["est_cost"]}
            p.free()
        res.append(row)
    return res


def root_work_tuples(G, n, queries, roots_per_query=2048, seed=0, time_limit_ms=30000, mem_bound=8 << 30):
    """Per-root training tuples: for each query (its Alg. 1-free connected order) and a
    stratified sample of roots, the features of huge_root_features and log(1 + work) with work =
    the EXTEND applications the enumerator makes from that root (the root and its partial
    matches at levels 1..k-2), logged by one batched launch with one root per plan copy."""
    import inputs

    X, Y = [], []
    rng = np.random.default_rng(seed)
    for qi, (k, e) in enumerate(queries):
        p = huge.Plan(G, k, e, order=random_connected_order(k, e, rng))
        m = min(n, roots_per_query)
        roots = np.minimum((np.arange(m) * (n / m) + inputs.uniform(m, 1 << 20, 7000 + seed * 1000 + qi)
                            / float(1 << 20) * (n / m)).astype(np.int64), n - 1).astype(np.uint32)
        lr = np.zeros((m, 16), dtype=np.int64)
        try:
            huge.enumerate_batch([p] * m, roots=[[int(r)] for r in roots], level_rows=lr,
                                 time_limit_ms=time_limit_ms, mem_bound=mem_bound)
        except huge.HugeError:
            p.free()
            continue
        work = 1.0 + lr[:, 1:k - 1].sum(axis=1).astype(np.float64)  # EXTEND applications from the root
        X.append(huge.root_features(p, roots))
        Y.append(np.log1p(work).astype(np.float32))
        p.free()
    return np.concatenate(X), np.concatenate(Y)


def root_partition_eval(G, n, queries, root_model, chunk_target=None, mem_bound=8 << 30):
    """Pre-partitioning roots by predicted work: device time of each query with root chunks
    balanced by (a) 1 + degree (the default) and (b) the root model's predicted work, both with
    work stealing off (the partition alone balances the warps) and, for reference, (c) the
    default with stealing on. Counts must be identical."""
    import torch

    res = []
    roots = np.arange(n, dtype=np.uint32)
    for k, e in queries:
        p = huge.Plan(G, k, e)
        X = huge.root_features(p, roots)
        pred = torch.zeros(n, dtype=torch.float32, device="cuda")
        dx = torch.from_numpy(X).cuda()
        root_model.forward(dx, pred)
        w = np.expm1(np.clip(pred.cpu().numpy(), 0, 60)).astype(np.float32)
        row = {"k": k, "edges": e, "order": p.describe().get("chain", {}).get("order")}
        for tag, kw in (("degree_nosteal", dict(flags=huge.EF_NO_STEAL)),
                        ("learned_nosteal", dict(flags=huge.EF_NO_STEAL, root_weights=w)),
                        ("degree_steal", dict()), ("learned_steal", dict(root_weights=w))):
            ts, c = [], None
            for _ in range(2):
                c, st = huge.enumerate(p, stats=True, mem_bound=mem_bound, **kw)
                ts.append(st["device_ms"])
            row[tag] = {"count": c, "device_ms": min(ts)}
        row["counts_identical"] = len({row[t]["count"] for t in ("degree_nosteal", "learned_nosteal",
                                                                  "degree_steal", "learned_steal")}) == 1
        res.append(row)
        p.free()
    return res


def connected_orders(k, edges):
    """Every matching order of the query whose prefixes are connected."""
    import itertools

    es = {tuple(x) for x in edges} | {(b, a) for a, b in edges}
    return [list(o) for o in itertools.permutations(range(k))
            if all(any((o[j], o[t]) in es for t in range(j)) for j in range(1, k))]


def regret_eval(G, queries, model, time_limit_ms=5000, mem_bound=8 << 30):
    """Plan regret of the plain and the learned estimator (EXTEND chains, automatic partial
    order). The true cost of a matching order is the sum of its exact intermediate result sizes
    |R(q'_i)| for the prefixes of 2..k-1 vertices (the partial matches the chain materialises,
    the quantity Alg. 1 minimises), read from the level counts of one exact enumeration per
    order; regret = cost of the chosen order / the smallest cost over every connected order."""
    out = []
    for k, e in queries:
        costs, count = {}, None
        for o in connected_orders(k, e):
            p = huge.Plan(G, k, e, order=o)
            try:
                c, st = huge.enumerate(p, stats=True, time_limit_ms=time_limit_ms, mem_bound=mem_bound)
                costs[tuple(o)] = float(sum(st["level_rows"][1:k]))
                count = c
            except huge.HugeError:
                costs[tuple(o)] = math.inf
            p.free()
        best = min(costs.values())
        row = {"k": k, "edges": e, "orders": len(costs), "best_cost": best, "count": count}
        for tag, flags, mdl in (("plain", huge.PLAN_EXTEND_ONLY, None),
                                ("learned", huge.PLAN_EXTEND_ONLY | huge.PLAN_LEARNED, model)):
            t0 = time.perf_counter()
            p = huge.Plan(G, k, e, flags=flags, model=mdl)
            t_plan = time.perf_counter() - t0
            order = tuple(p.describe()["chain"]["order"])
            p.free()
            row[tag] = {"order": list(order), "plan_s": t_plan, "cost": costs[order],
                        "regret": costs[order] / best if best > 0 else 1.0}
        out.append(row)
    return out


def main():
    import inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("--tuples", type=int, default=50000)
    ap.add_argument("--budget-s", type=float, default=300)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--out", default="")
    ap.add_argument("--model", default="")
    ap.add_argument("--regret-scale", type=int, default=16)
    ap.add_argument("--regret-limit-ms", type=int, default=5000)
    ap.add_argument("--root-model", action="store_true", help="train and evaluate the per-root work model")
    ap.add_argument("--root-scale", type=int, default=20)
    ap.add_argument("--regret-queries", type=int, default=12)
    ap.add_argument("--eval-scale", type=int, default=23)
    ap.add_argument("--collect-limit-ms", type=int, default=200)
    ap.add_argument("--eval-queries", type=int, default=8)
    ap.add_argument("--eval-limit-ms", type=int, default=60000)
    args = ap.parse_args()
    report = {}
    if args.model:
        model = load_model(args.model)
    else:
        # training graphs: R-MAT scales 12-16 and Chung-Lu graphs small enough that exact runs of
        # 3-6-vertex queries finish in milliseconds (many tuples per second)
        graphs, kmax = [], {}
        for s in (12, 13, 14, 15, 16):
            name = f"rmat{s}"
            g = inputs.rmat(s, 16, 100 + s)
            graphs.append((name, huge.Graph(g.offsets, g.adj)))
            kmax[name] = 6 if s <= 12 else (5 if s <= 14 else 4)
        for lg in (13, 15, 16):
            name = f"chunglu{1 << lg}"
            n = 1 << lg
            g = inputs.chung_lu(n, 8 * n, 200 + lg, max_w=float(n) ** 0.6)
            graphs.append((name, huge.Graph(g.offsets, g.adj)))
            kmax[name] = 6 if lg <= 13 else 5
        t0 = time.time()
        X, Y, meta = collect_batched(graphs, args.tuples, seed=1, budget_s=args.budget_s, verbose=True, kmax=kmax)
        t_collect = time.time() - t0
        t0 = time.time()
        model, loss, rmse = train(X, Y, epochs=args.epochs)
        report["training"] = {"tuples": int(len(Y)), "collect_s": t_collect, "train_s": time.time() - t0,
                              "final_loss": loss, "holdout_rmse_log": rmse, "label_std_log": float(np.std(Y)),
                              "graphs": [n for n, _ in graphs]}
        if args.out:
            save(model, args.out)
        for _, G in graphs:
            G.free()
        print(json.dumps({"training": report["training"]}), flush=True)  # each part as it completes
    if args.root_model:
        # the per-root work model: tuples on R-MAT 14-16, evaluated on the benchmark graph
        import torch  # noqa: F401

        tX, tY = [], []
        for sc in (14, 15, 16):
            g = inputs.rmat(sc, 16, 400 + sc)
            G = huge.Graph(g.offsets, g.adj)
            qs = [inputs.QUERIES[nm] for nm in ("k4", "c4", "diamond", "tailed_triangle", "triangle")]
            qs += [inputs.random_query(3 + (s % 3), 500 + s) for s in range(6)]
            x, y = root_work_tuples(G, g.n, qs, seed=sc)
            tX.append(x)
            tY.append(y)
            G.free()
        X, Y = np.concatenate(tX), np.concatenate(tY)
        t0 = time.time()
        rmodel, rloss, rrmse = train(X, Y, epochs=args.epochs)
        g = inputs.rmat(args.root_scale, 16, 2)
        G = huge.Graph(g.offsets, g.adj)
        rows = root_partition_eval(G, g.n, [inputs.QUERIES[nm] for nm in ("k4", "c4")], rmodel)
        report["root_partition"] = {"tuples": int(len(Y)), "train_s": time.time() - t0, "holdout_rmse_log": rrmse,
                                    "label_std_log": float(np.std(Y)), "eval_graph": f"rmat{args.root_scale}-ef16-s2",
                                    "queries": rows}
        G.free()
        print(json.dumps({"root_partition": report["root_partition"]}), flush=True)
    if args.regret_scale:
        g = inputs.rmat(args.regret_scale, 16, 60)
        G = huge.Graph(g.offsets, g.adj)
        queries = [inputs.random_query(4 + (s % 2), 900 + s) for s in range(args.regret_queries)]
        rows = regret_eval(G, queries, model, time_limit_ms=args.regret_limit_ms)
        fin = [r for r in rows if math.isfinite(r["best_cost"])]
        report["regret"] = {"graph": f"rmat{args.regret_scale}-ef16-s60", "queries": rows,
                            "mean_regret_plain": float(np.mean([r["plain"]["regret"] for r in fin])) if fin else None,
                            "mean_regret_learned": float(np.mean([r["learned"]["regret"] for r in fin])) if fin else None,
                            "plan_s_plain": float(sum(r["plain"]["plan_s"] for r in rows)),
                            "plan_s_learned": float(sum(r["learned"]["plan_s"] for r in rows))}
        G.free()
        print(json.dumps({"regret": report["regret"]}), flush=True)
    if args.eval_scale:
        g = inputs.rmat(args.eval_scale, 16, 50)
        G = huge.Graph(g.offsets, g.adj, flags=huge.RELABEL_BY_DEGREE | huge.TRUST_SORTED)
        queries = []
        s = 50
        while len(queries) < args.eval_queries:
            k = 4 + (s % 2)  # 4- and 5-vertex queries, denser (extra pairs w.p. 3/4) so that runs finish
            queries.append(inputs.random_query(k, s, 3, 4))
            s += 1
        res = compare(G, queries, model, time_limit_ms=args.eval_limit_ms)
        done = [r for r in res if r["plain"]["count"] is not None and r["learned"]["count"] is not None]
        report["eval"] = {"graph": f"rmat{args.eval_scale}-ef16-s50", "n": g.n, "m": g.m, "queries": res,
                          "finished_both": len(done),
                          "counts_identical": all(r["plain"]["count"] == r["learned"]["count"] for r in done),
                          "e2e_s_plain": float(sum(r["plain"]["e2e_s"] for r in done)),
                          "e2e_s_learned": float(sum(r["learned"]["e2e_s"] for r in done))}
    print(json.dumps(report))


if __name__ == "__main__":
    main()
