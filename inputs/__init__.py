"""Seeded synthetic inputs shared by the CUDA path's tests and the CPU oracle.

Only input generation lives here: random data graphs in simple undirected CSR form (sorted
adjacency, no self-loops, no duplicates) and query graphs. Nothing in this module computes
any part of the enumeration method (no relabelling, no intersections, no partial orders).

The C generators in ``gen.c`` are built into ``libgen.so`` beside this file on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgen.so")
_SRC = os.path.join(_HERE, "gen.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so (gcc, OpenMP). Returns the library path."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.POINTER(ctypes.c_uint64))
            u32p = ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))
            lib.gen_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u64p, u32p]
            lib.gen_gnp.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint64, u64p, u32p]
            lib.gen_complete.argtypes = [ctypes.c_uint32, u64p, u32p]
            lib.gen_complete_bipartite.argtypes = [ctypes.c_uint32, ctypes.c_uint32, u64p, u32p]
            lib.gen_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_uint64, u64p, u32p]
            lib.gen_rmat_directed.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_uint64, u64p, u32p]
            lib.gen_gnp_directed.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint64, u64p, u32p]
            lib.gen_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_uint64, u64p, u32p]
            lib.gen_random_query.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32)]
            lib.gen_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_uint64)]
            lib.gen_free.argtypes = [ctypes.c_void_p]
            _lib = lib
    return _lib


class Graph:
    """A simple undirected graph in CSR form: ``offsets`` (uint64, n+1) and ``adj`` (uint32)."""

    def __init__(self, offsets: np.ndarray, adj: np.ndarray, name: str = ""):
        self.offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        self.adj = np.ascontiguousarray(adj, dtype=np.uint32)
        self.name = name

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)

    def __repr__(self) -> str:
        return f"Graph({self.name!r}, n={self.n}, m={self.m})"


def _call(fn, *args, n: int, name: str) -> Graph:
    lib = _load()
    po = ctypes.POINTER(ctypes.c_uint64)()
    pa = ctypes.POINTER(ctypes.c_uint32)()
    rc = fn(*args, ctypes.byref(po), ctypes.byref(pa))
    if rc != 0:
        raise ValueError(f"generator {name} failed (rc={rc})")
    offsets = np.ctypeslib.as_array(po, shape=(n + 1,)).copy()
    nnz = int(offsets[-1])
    adj = np.ctypeslib.as_array(pa, shape=(max(nnz, 1),))[:nnz].copy()
    lib.gen_free(ctypes.cast(po, ctypes.c_void_p))
    lib.gen_free(ctypes.cast(pa, ctypes.c_void_p))
    return Graph(offsets, adj, name)


def er(n: int, m: int, seed: int) -> Graph:
    """Erdos-Renyi G(n, m): m distinct unordered pairs drawn uniformly (no loops)."""
    return _call(_load().gen_er, n, m, seed, n=n, name=f"er-{n}-{m}-s{seed}")


def gnp(n: int, p_num: int, p_den: int, seed: int) -> Graph:
    """Erdos-Renyi G(n, p) with p = p_num / p_den, for tiny graphs."""
    return _call(_load().gen_gnp, n, p_num, p_den, seed, n=n, name=f"gnp-{n}-{p_num}/{p_den}-s{seed}")


def complete(n: int) -> Graph:
    return _call(_load().gen_complete, n, n=n, name=f"K{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    return _call(_load().gen_complete_bipartite, a, b, n=a + b, name=f"K{a},{b}")


def rmat(scale: int, edge_factor: int, seed: int, a: float = 0.57, b: float = 0.19,
         c: float = 0.19) -> Graph:
    """R-MAT without noise, self-loops dropped, symmetrised and deduplicated (ids unpermuted)."""
    return _call(_load().gen_rmat, scale, edge_factor, a, b, c, seed, n=1 << scale,
                 name=f"rmat-{scale}-ef{edge_factor}-s{seed}")


def rmat_directed(scale: int, edge_factor: int, seed: int, a: float = 0.57, b: float = 0.19,
                  c: float = 0.19) -> Graph:
    """Directed R-MAT: the samples kept as arcs (self-loops dropped, repeats merged); CSR of
    out-lists, not symmetric."""
    return _call(_load().gen_rmat_directed, scale, edge_factor, a, b, c, seed, n=1 << scale,
                 name=f"rmat-directed-{scale}-ef{edge_factor}-s{seed}")


def gnp_directed(n: int, p_num: int, p_den: int, seed: int) -> Graph:
    """Directed G(n, p): each ordered pair u != v is an arc with probability p_num / p_den."""
    return _call(_load().gen_gnp_directed, n, p_num, p_den, seed, n=n, name=f"dgnp-{n}-{p_num}/{p_den}-s{seed}")


def chung_lu(n: int, m: int, seed: int, gamma: float = 2.1, max_w: float = 15000.0) -> Graph:
    """Chung-Lu power-law graph with exactly m distinct undirected edges."""
    return _call(_load().gen_chung_lu, n, m, gamma, max_w, seed, n=n,
                 name=f"chunglu-{n}-{m}-s{seed}")


def random_query(k: int, seed: int, p_num: int = 1, p_den: int = 2):
    """Random connected query graph on k vertices: random spanning tree + each other pair
    with probability p_num/p_den. Returns (k, [(u, v), ...])."""
    lib = _load()
    buf = (ctypes.c_uint32 * (k * (k - 1)))()
    mq = lib.gen_random_query(k, p_num, p_den, seed, buf)
    if mq < 0:
        raise ValueError("bad query size")
    return k, [(int(buf[2 * i]), int(buf[2 * i + 1])) for i in range(mq)]


def uniform(count: int, n: int, seed: int) -> np.ndarray:
    """`count` seeded uniform integers in [0, n)."""
    out = np.zeros(max(count, 1), dtype=np.uint64)
    _load().gen_uniform(count, n, seed, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out[:count]


# Named query graphs (vertex count, edge list). The paper's own q1-q8 exist only in a figure
# that is not available; these are the shapes the workloads name.
QUERIES = {
    "triangle": (3, [(0, 1), (1, 2), (0, 2)]),
    "k4": (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
    "c4": (4, [(0, 1), (1, 2), (2, 3), (3, 0)]),
    "k5": (5, [(u, v) for u in range(5) for v in range(u + 1, 5)]),
    # square 0-1-2-3-0 with a roof vertex 4 adjacent to 0 and 1 (4-cycle + triangle on edge 01)
    "house": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (1, 4)]),
    # diamond = K4 minus edge {2,3}; pendant tail vertex 4 attached to vertex 2 (degree 2)
    "tailed_diamond_a": (5, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 4)]),
    "path3": (3, [(0, 1), (1, 2)]),
    "path4": (4, [(0, 1), (1, 2), (2, 3)]),
    "path5": (5, [(0, 1), (1, 2), (2, 3), (3, 4)]),
    "star4": (4, [(0, 1), (0, 2), (0, 3)]),
    "c5": (5, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]),
    "c6": (6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0)]),
    "diamond": (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)]),
    "tailed_triangle": (4, [(0, 1), (1, 2), (0, 2), (2, 3)]),
}

# Workload recipes (seeds and sizes) for the five synthetic workloads.
WORKLOADS = {
    "er2000": dict(kind="er", n=2000, m=20000, seed=1),
    "rmat20": dict(kind="rmat", scale=20, edge_factor=16, seed=2),
    "chunglu4m": dict(kind="chung_lu", n=4 * 1024 * 1024, m=35_000_000, seed=3),
    # the Chung-Lu recipe at 1/64 of the vertices and edges (hubs up to ~700), small enough
    # for whole-graph CPU counts of the 5-vertex queries
    "chunglu64k": dict(kind="chung_lu", n=65536, m=546_875, seed=3, max_w=700.0),
    "rmat22": dict(kind="rmat", scale=22, edge_factor=16, seed=4),
    "rmat23": dict(kind="rmat", scale=23, edge_factor=16, seed=50),
}


def workload_graph(name: str, **over) -> Graph:
    spec = dict(WORKLOADS[name])
    spec.update(over)
    kind = spec.pop("kind")
    if kind == "er":
        return er(spec["n"], spec["m"], spec["seed"])
    if kind == "rmat":
        return rmat(spec["scale"], spec["edge_factor"], spec["seed"])
    if kind == "chung_lu":
        return chung_lu(spec["n"], spec["m"], spec["seed"], max_w=spec.get("max_w", 15000.0))
    raise KeyError(kind)
