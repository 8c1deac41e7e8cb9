"""Alg. 5, the DFS/BFS-adaptive scheduler, as a plain host model — TEST INFRASTRUCTURE ONLY.

Like the rest of ``oracle``, only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
legs of ``bench.py`` may import this module; the library never does, and nothing here comes
from it.

A dataflow is a chain of operators, SCAN first and SINK last, EXTENDs between (Sec. 4.2).
Every operator but SINK owns an output queue of at most ``cap`` batches, which is the next
operator's input (Sec. 5.2). The scheduler of Alg. 5 works as follows:

* Scheduling an operator lets it consume its input one batch at a time, appending what each
  batch produces to its output queue.
* It yields once the queue is full or its input is empty (the check comes before every batch).
* After SINK it moves to the precursor (backtracking); after any other operator, to the
  successor.
* An operator other than SCAN that has no input hands control to its precursor without being
  scheduled.
* SCAN's input is the data graph itself, cut into source units.
* The run ends when no operator has work left.

``run`` records which operator every scheduling slot ran and the longest each queue grew. With
those records, tests can check two things:

* the running example of the scheduler in Sec. 5.2, slot by slot;
* the memory bound of Sec. 5.2 on real data. A queue never holds more than ``cap - 1``
  batches plus the batches one input batch can produce.

``extend_ops`` builds the operators of a matching order from the definition of a match
(Sec. 2): EXTEND binds the next query vertex to a common neighbour of its bound query
neighbours, distinct from the bound vertices and inside the partial order's bounds (Eq. 2,
Alg. 4). The SINK's rows are then exactly the matches that ``oracle.count`` counts.
"""
from __future__ import annotations


def run(source, ops, cap: int, max_slots: int = 10_000_000):
    """Alg. 5 over a chain of len(ops) >= 2 operators.

    source: the SCAN's source units (a list). ops[0](unit) -> list of batches is the SCAN,
    ops[i](batch) -> list of batches the EXTENDs, and ops[-1](batch) the SINK (its return value
    is collected). cap: output-queue capacity in batches (>= 1).

    Returns a dict:
      trace: the operator index of every scheduling slot, in order;
      peak: the longest each output queue grew (in batches; the SINK's entry is 0);
      sink: whatever the SINK returned, batch by batch.
    """
    if cap < 1 or len(ops) < 2:
        raise ValueError("need cap >= 1 and at least a SCAN and a SINK")
    L = len(ops)
    src = list(source)
    queues = [[] for _ in range(L - 1)]  # queues[i]: output of operator i = input of i + 1
    peak = [0] * L
    trace, sink = [], []

    def has_input(i):
        return bool(src) if i == 0 else bool(queues[i - 1])

    def done():  # every queue drained and the source exhausted
        return not src and not any(queues)

    o = 0
    while not done():
        if not has_input(o) and o != 0:
            o -= 1  # precursor
            continue
        if len(trace) >= max_slots:
            raise RuntimeError("no progress within max_slots scheduling slots")
        trace.append(o)
        while True:  # Schedule(O) until its queue is full or its input is empty, then Yield(O)
            full = o < L - 1 and len(queues[o]) >= cap
            if full or not has_input(o):
                break
            item = src.pop(0) if o == 0 else queues[o - 1].pop(0)
            out = ops[o](item)
            if o == L - 1:
                sink.append(out)
            else:
                queues[o].extend(out)
                peak[o] = max(peak[o], len(queues[o]))
        o = o - 1 if o == L - 1 else o + 1
    return {"trace": trace, "peak": peak, "sink": sink}


def _batches(rows, b):
    return [rows[i:i + b] for i in range(0, len(rows), b)]


def extend_ops(adj, k: int, edges, order, po=(), batch_rows: int = 4):
    """SCAN, EXTENDs and a counting SINK for matching order `order` of query (k, edges) on
    data graph `adj` (a list of neighbour sets), with partial-order pairs `po` (a, b meaning
    f(a) < f(b)). Rows hold the data vertices bound to order[0], order[1], ... Source units are
    single root vertices; every operator cuts its output into batches of `batch_rows` rows.
    Returns (source, ops)."""
    qn = {v: set() for v in range(k)}
    for a, b in edges:
        qn[a].add(b)
        qn[b].add(a)
    pos = {v: j for j, v in enumerate(order)}
    lt = set(map(tuple, po))
    for j in range(1, k):
        if not qn[order[j]] & set(order[:j]):
            raise ValueError("every prefix of the matching order must be connected")

    def ok(row, u, j):  # injective and inside the partial order's bounds at position j
        v = order[j]
        for t in range(j):
            w = order[t]
            if row[t] == u:
                return False
            if (w, v) in lt and not row[t] < u:
                return False
            if (v, w) in lt and not u < row[t]:
                return False
        return True

    def scan(r):  # rows (r, u1): u1 a neighbour of r that may take order[1]
        return _batches([(r, u) for u in sorted(adj[r]) if ok((r,), u, 1)], batch_rows)

    def make_extend(j):
        nb = [pos[w] for w in qn[order[j]] if pos[w] < j]

        def extend(batch):
            out = []
            for row in batch:
                cand = set.intersection(*[adj[row[p]] for p in nb])
                out.extend(row + (u,) for u in sorted(cand) if ok(row, u, j))
            return _batches(out, batch_rows)

        return extend

    ops = [scan] + [make_extend(j) for j in range(2, k)] + [len]
    return list(range(len(adj))), ops
