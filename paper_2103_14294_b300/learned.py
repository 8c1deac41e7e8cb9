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


def main():
    import inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("--tuples", type=int, default=50000)
    ap.add_argument("--budget-s", type=float, default=600)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--out", default="")
    ap.add_argument("--model", default="")
    ap.add_argument("--eval-scale", type=int, default=23)
    ap.add_argument("--collect-limit-ms", type=int, default=60)
    ap.add_argument("--eval-queries", type=int, default=8)
    ap.add_argument("--eval-limit-ms", type=int, default=60000)
    args = ap.parse_args()
    report = {}
    if args.model:
        model = load_model(args.model)
    else:
        graphs, kmax = [], {}
        for s in (16, 16, 17, 17, 18, 19, 20):
            name = f"rmat{s}-{len(graphs)}"
            g = inputs.rmat(s, 16, 100 + len(graphs))
            graphs.append((name, huge.Graph(g.offsets, g.adj)))
            kmax[name] = 6 if s <= 17 else (5 if s == 18 else 4)
        for n in (1 << 16, 1 << 18):
            name = f"chunglu{n}"
            g = inputs.chung_lu(n, 8 * n, 200 + n.bit_length())
            graphs.append((name, huge.Graph(g.offsets, g.adj)))
            kmax[name] = 6 if n <= 1 << 16 else 5
        t0 = time.time()
        X, Y, meta = collect(graphs, args.tuples, seed=1, time_limit_ms=args.collect_limit_ms,
                             budget_s=args.budget_s, verbose=True, kmax=kmax)
        t_collect = time.time() - t0
        t0 = time.time()
        model, loss, rmse = train(X, Y, epochs=args.epochs)
        report["training"] = {"tuples": int(len(Y)), "collect_s": t_collect, "train_s": time.time() - t0,
                              "final_loss": loss, "holdout_rmse_log": rmse,
                              "graphs": [n for n, _ in graphs]}
        if args.out:
            save(model, args.out)
        for _, G in graphs:
            G.free()
    if args.eval_scale:
        g = inputs.rmat(args.eval_scale, 16, 50)
        G = huge.Graph(g.offsets, g.adj, flags=huge.RELABEL_BY_DEGREE | huge.TRUST_SORTED)
        queries = []
        for s in range(50, 50 + args.eval_queries):
            k = 4 + (s % 2)  # 4- and 5-vertex queries
            queries.append(inputs.random_query(k, s))
        res = compare(G, queries, model, time_limit_ms=args.eval_limit_ms)
        report["eval"] = {"graph": f"rmat{args.eval_scale}-ef16-s50", "n": g.n, "m": g.m, "queries": res}
    print(json.dumps(report))


if __name__ == "__main__":
    main()
