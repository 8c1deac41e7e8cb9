"""Thin ctypes binding of libhuge.so (include/huge.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. PyTorch is used only for device memory
(LIST sinks, MLP tensors) and streams. Loading fails loudly if the library is missing: there is
no fallback path.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhuge.so")

OK, EINVAL, ENOMEM, EOVERFLOW, ETIMEOUT, ECUDA, ERANGE = 0, 1, 2, 3, 4, 5, 6
RELABEL_BY_DEGREE, TRUST_SORTED, DIRECTED = 1, 2, 4
ANY_LABEL = 0xFFFFFFFF
PLAN_PLAIN, PLAN_LEARNED, PLAN_EXTEND_ONLY, PLAN_TREE_VERIFY, PLAN_FORCE_JOIN = 0, 1, 2, 4, 8
PLAN_DIRECTED = 16
COUNT, LIST = 0, 1
EF_STATS, EF_NO_STEAL = 1, 2
MAX_QUERY_VERTICES = 8

_ERRNAMES = {EINVAL: "HUGE_EINVAL", ENOMEM: "HUGE_ENOMEM", EOVERFLOW: "HUGE_EOVERFLOW",
             ETIMEOUT: "HUGE_ETIMEOUT", ECUDA: "HUGE_ECUDA", ERANGE: "HUGE_ERANGE"}


class HugeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


DRAIN_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64)


class Sink(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_void_p), ("capacity_rows", ctypes.c_uint64), ("drain", DRAIN_FN),
                ("ctx", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("level_rows", ctypes.c_int64 * 16), ("nlevels", ctypes.c_int32),
                ("intersections", ctypes.c_uint64), ("list_bytes", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64), ("device_ms", ctypes.c_double),
                ("level_cap", ctypes.c_uint32), ("warps", ctypes.c_uint32), ("launches", ctypes.c_uint32)]

    def as_dict(self):
        return {"level_rows": list(self.level_rows[: self.nlevels]), "intersections": self.intersections,
                "list_bytes": self.list_bytes, "peak_bytes": self.peak_bytes, "device_ms": self.device_ms,
                "level_cap": self.level_cap, "warps": self.warps, "launches": self.launches}


class EnumOpts(ctypes.Structure):
    _fields_ = [("root_begin", ctypes.c_uint32), ("root_end", ctypes.c_uint32),
                ("roots", ctypes.c_void_p), ("nroots", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("level_cap", ctypes.c_uint32), ("chunk_roots", ctypes.c_uint32),
                ("root_weights", ctypes.c_void_p), ("time_limit_ms", ctypes.c_uint32),
                ("variant", ctypes.c_uint32), ("per_root", ctypes.c_void_p)]


_lib = None

# (name, restype, argtypes) of every exported function
_P = ctypes.c_void_p
_SIGS = [
    ("huge_last_error", ctypes.c_char_p, []),
    ("huge_graph_load", ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, _P]),
    ("huge_graph_free", ctypes.c_int, [_P]),
    ("huge_graph_load_labeled", ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.c_uint64, _P, ctypes.c_uint32,
                                               ctypes.c_uint32, _P]),
    ("huge_graph_label_ranges", ctypes.c_int, [_P, _P, _P]),
    ("huge_plan_labeled", ctypes.c_int, [_P, ctypes.c_uint32, _P, ctypes.c_uint32, _P, _P, _P, ctypes.c_int32,
                                         ctypes.c_uint32, _P, _P]),
    ("huge_graph_info", ctypes.c_int, [_P, _P, _P, _P]),
    ("huge_graph_new_ids", ctypes.c_int, [_P, _P]),
    ("huge_graph_set_hub_bitmaps", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64]),
    ("huge_graph_hub_info", ctypes.c_int, [_P, _P, _P, _P]),
    ("huge_graph_set_residency", ctypes.c_int, [_P, ctypes.c_uint64, _P]),
    ("huge_plan", ctypes.c_int, [_P, ctypes.c_uint32, _P, ctypes.c_uint32, _P, _P, ctypes.c_int32,
                                 ctypes.c_uint32, _P]),
    ("huge_plan_ex", ctypes.c_int, [_P, ctypes.c_uint32, _P, ctypes.c_uint32, _P, _P, ctypes.c_int32,
                                    ctypes.c_uint32, _P, _P]),
    ("huge_plan_free", ctypes.c_int, [_P]),
    ("huge_plan_describe", ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_size_t]),
    ("huge_plan_timing", ctypes.c_int, [_P, _P, _P]),
    ("huge_plan_offline", ctypes.c_int, [ctypes.c_uint32, _P, ctypes.c_uint32, _P, _P, ctypes.c_int32,
                                         ctypes.c_uint32, _P, ctypes.c_double, ctypes.c_char_p, ctypes.c_size_t]),
    ("huge_plan_offline_labeled", ctypes.c_int, [ctypes.c_uint32, _P, ctypes.c_uint32, _P, _P, ctypes.c_uint32, _P,
                                                 _P, ctypes.c_int32, ctypes.c_uint32, _P, ctypes.c_double,
                                                 ctypes.c_char_p, ctypes.c_size_t]),
    ("huge_enumerate", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint64, _P, _P, _P]),
    ("huge_enumerate_ex", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint64, _P, _P, _P, _P, _P]),
    ("huge_enumerate_batch", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, _P, _P, _P]),
    ("huge_enumerate_batch_ex", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, _P, _P, _P, _P, _P]),
    ("huge_autotune", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, _P, _P, _P]),
    ("huge_mlp_num_params", ctypes.c_uint32, []),
    ("huge_mlp_create", ctypes.c_int, [ctypes.c_uint64, _P]),
    ("huge_mlp_free", ctypes.c_int, [_P]),
    ("huge_mlp_set_params", ctypes.c_int, [_P, _P, _P, _P]),
    ("huge_mlp_get_params", ctypes.c_int, [_P, _P, _P, _P]),
    ("huge_mlp_forward", ctypes.c_int, [_P, _P, ctypes.c_uint32, _P, _P]),
    ("huge_mlp_loss_grad", ctypes.c_int, [_P, _P, _P, ctypes.c_uint32, _P, _P, _P]),
    ("huge_mlp_train", ctypes.c_int, [_P, _P, _P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_float, _P, _P]),
    ("huge_plan_features", ctypes.c_int, [_P, ctypes.c_uint32, _P, ctypes.c_uint32, _P, ctypes.c_int32,
                                          ctypes.c_uint32, _P]),
    ("huge_count_noalloc", ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, _P,
                                          ctypes.c_uint32, _P, _P, ctypes.c_int32, _P, _P]),
    ("huge_set_allocator", ctypes.c_int, [_P, _P, _P]),
    ("huge_root_features", ctypes.c_int, [_P, _P, ctypes.c_uint64, _P]),
]

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int)
_hooks = None  # the ctypes callbacks must outlive every block they made


def _torch_alloc(ctx, nbytes, device):
    try:
        import torch

        return torch.cuda.caching_allocator_alloc(int(nbytes), device=int(device))
    except Exception:  # out of memory or torch unavailable: the library reports HUGE_ENOMEM
        return None


def _torch_free(ctx, ptr, device):
    try:
        import torch

        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:  # interpreter shutdown: the process is ending anyway
        pass


def use_torch_allocator(enable: bool = True):
    """Routes the library's device buffers through PyTorch's caching allocator (the hook of
    huge_set_allocator), or back to cudaMalloc."""
    global _hooks
    lib = load()
    if enable:
        if _hooks is None:
            _hooks = (ALLOC_FN(_torch_alloc), FREE_FN(_torch_free))
        _check(lib.huge_set_allocator(ctypes.cast(_hooks[0], ctypes.c_void_p),
                                      ctypes.cast(_hooks[1], ctypes.c_void_p), None))
    else:
        _check(lib.huge_set_allocator(None, None, None))


def exported_names():
    return [s[0] for s in _SIGS]


def load(path: str | None = None):
    """Loads libhuge.so (raises if it is missing: no fallback)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library {p} is missing; build it with "
                               "`python -m paper_2103_14294_b300.build` (no CPU fallback exists)")
        lib = ctypes.CDLL(p)
        for name, res, args in _SIGS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        if os.environ.get("HUGE_TORCH_ALLOCATOR", "1") != "0":
            try:
                import torch

                torch_cuda = torch.cuda.is_available()
            except ImportError:
                torch_cuda = False
            if torch_cuda:
                use_torch_allocator(True)
    return _lib


def _check(rc: int):
    if rc != OK:
        raise HugeError(rc, load().huge_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _need_host(a, count: int, name: str):
    """The C side reads `count` entries of a host array through a plain pointer."""
    if a is not None and len(a) < count:
        raise HugeError(EINVAL, f"{name} holds {len(a)} entries, needs {count}")


def _need_device(t, count: int, name: str, dtypes=("float32",), width: int | None = None):
    """A CUDA tensor the C side reads or writes `count` entries of (a raw device address is
    passed through unchecked): contiguous, of the given dtype, on the current device."""
    if not hasattr(t, "data_ptr"):
        return
    import torch

    if str(t.dtype).replace("torch.", "") not in dtypes or not t.is_contiguous():
        raise HugeError(EINVAL, f"{name} must be a contiguous {'/'.join(dtypes)} tensor")
    if width is not None and (t.dim() != 2 or t.shape[1] != width):
        raise HugeError(EINVAL, f"{name} must have shape (rows, {width})")
    if t.numel() < count:
        raise HugeError(EINVAL, f"{name} holds {t.numel()} entries, needs {count}")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise HugeError(EINVAL, f"{name} must be on the current CUDA device")


class Graph:
    """A data graph loaded onto the device (huge_graph_load)."""

    def __init__(self, offsets, adj, n: int | None = None, flags: int = RELABEL_BY_DEGREE, labels=None,
                 nlabels: int | None = None):
        """labels: optional vertex labels (n entries, original ids) -> huge_graph_load_labeled."""
        lib = load()
        self._offsets = np.ascontiguousarray(offsets, dtype=np.uint64).ravel()
        self._adj = np.ascontiguousarray(adj, dtype=np.uint32).ravel()
        # the C side reads offsets[0..n] and adj[0..offsets[n]) through plain pointers: check
        # that the arrays hold them
        n = len(self._offsets) - 1 if n is None else int(n)
        if n < 0 or len(self._offsets) < n + 1:
            raise HugeError(EINVAL, f"offsets holds {len(self._offsets)} entries, needs n + 1 = {n + 1}")
        nnz = int(self._offsets[n])
        if len(self._adj) < nnz:
            raise HugeError(EINVAL, f"adj holds {len(self._adj)} entries, offsets[n] = {nnz}")
        h = ctypes.c_void_p()
        if labels is None:
            _check(lib.huge_graph_load(_ptr(self._offsets), _ptr(self._adj), n, nnz, flags, ctypes.byref(h)))
        else:
            lab = np.ascontiguousarray(labels, dtype=np.uint32).ravel()
            if len(lab) < n:
                raise HugeError(EINVAL, f"labels holds {len(lab)} entries, needs n = {n}")
            nl = (int(lab.max()) + 1 if len(lab) else 1) if nlabels is None else int(nlabels)
            _check(lib.huge_graph_load_labeled(_ptr(self._offsets), _ptr(self._adj), n, nnz, _ptr(lab), nl, flags,
                                               ctypes.byref(h)))
        self.handle = h
        self._offsets = self._adj = None

    def label_ranges(self):
        """[lstart[0], ..., lstart[L]]: label l owns the library's ids [lstart[l], lstart[l+1])."""
        nl = ctypes.c_uint32()
        _check(load().huge_graph_label_ranges(self.handle, ctypes.byref(nl), None))
        out = np.zeros(nl.value + 1, dtype=np.uint32)
        if nl.value:
            _check(load().huge_graph_label_ranges(self.handle, ctypes.byref(nl), _ptr(out)))
        return out[: nl.value + 1] if nl.value else out[:0]

    def info(self):
        n, nnz, md = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint32()
        _check(load().huge_graph_info(self.handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(md)))
        return {"n": n.value, "nnz": nnz.value, "max_degree": md.value}

    def set_hub_bitmaps(self, min_degree: int | None = None, max_bytes: int = 4 << 30):
        """(Re)builds the hub adjacency bitmaps (huge_graph_set_hub_bitmaps); min_degree None
        selects the library default, 0 removes them."""
        md = 0xFFFFFFFF if min_degree is None else int(min_degree)
        _check(load().huge_graph_set_hub_bitmaps(self.handle, md, int(max_bytes)))

    def set_residency(self, hbm_bytes: int) -> int:
        """Keeps the last hbm_bytes of the adjacency in HBM, the rest in host memory
        (huge_graph_set_residency); returns the adjacency bytes resident in HBM."""
        out = ctypes.c_uint64()
        _check(load().huge_graph_set_residency(self.handle, min(int(hbm_bytes), (1 << 64) - 1), ctypes.byref(out)))
        return out.value

    def hub_info(self):
        c, md, b = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
        _check(load().huge_graph_hub_info(self.handle, ctypes.byref(c), ctypes.byref(md), ctypes.byref(b)))
        return {"count": c.value, "min_degree": md.value, "bytes": b.value}

    def new_ids(self) -> np.ndarray:
        out = np.zeros(self.info()["n"], dtype=np.uint32)
        _check(load().huge_graph_new_ids(self.handle, _ptr(out)))
        return out

    def free(self):
        if self.handle:
            load().huge_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Plan:
    """An execution plan (huge_plan / huge_plan_ex)."""

    def __init__(self, graph: Graph, k: int, edges, order=None, po=None, flags: int = PLAN_PLAIN, model=None,
                 labels=None):
        """labels: optional query vertex labels (k entries, ANY_LABEL = any) -> huge_plan_labeled."""
        lib = load()
        e = np.asarray([x for uv in edges for x in uv] or [0], dtype=np.uint32)
        o = None if order is None else np.asarray(order, dtype=np.uint32)
        _need_host(o, k, "order")
        if po is None:
            pa, npo = None, -1
        else:
            pa = np.asarray([x for ab in po for x in ab] or [0], dtype=np.uint32)
            npo = len(po)
        h = ctypes.c_void_p()
        mh = model.handle if model is not None else None
        if labels is None:
            _check(lib.huge_plan_ex(graph.handle, k, _ptr(e), len(edges), _ptr(o), _ptr(pa), npo, flags, mh,
                                    ctypes.byref(h)))
        else:
            ql = np.ascontiguousarray(labels, dtype=np.uint32)
            _need_host(ql, k, "labels")
            _check(lib.huge_plan_labeled(graph.handle, k, _ptr(e), len(edges), _ptr(ql), _ptr(o), _ptr(pa), npo,
                                         flags, mh, ctypes.byref(h)))
        self.handle = h
        self.graph = graph
        self.k = k

    def describe(self) -> dict:
        buf = ctypes.create_string_buffer(16384)
        _check(load().huge_plan_describe(self.handle, buf, len(buf)))
        return json.loads(buf.value.decode())

    def timing(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(load().huge_plan_timing(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def free(self):
        if self.handle:
            load().huge_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def plan_offline(k: int, edges, order=None, po=None, flags: int = PLAN_PLAIN, card=None,
                 edges_g: float = 0.0, labels=None, lstart=None) -> dict:
    """huge_plan_offline(_labeled): the planner alone on the host (no graph, no GPU). card: 2**k
    cardinality estimates indexed by vertex mask (needed when order is None); labels / lstart: a
    labelled query and the label ranges of its graph."""
    lib = load()
    e = np.asarray([x for uv in edges for x in uv] or [0], dtype=np.uint32)
    o = None if order is None else np.asarray(order, dtype=np.uint32)
    _need_host(o, k, "order")
    if po is None:
        pa, npo = None, -1
    else:
        pa = np.asarray([x for ab in po for x in ab] or [0], dtype=np.uint32)
        npo = len(po)
    c = None if card is None else np.ascontiguousarray(card, dtype=np.float64)
    if c is not None and len(c) != 1 << k:
        raise ValueError("card needs 2**k entries")
    buf = ctypes.create_string_buffer(65536)
    if labels is None:
        _check(lib.huge_plan_offline(k, _ptr(e), len(edges), _ptr(o), _ptr(pa), npo, flags, _ptr(c), float(edges_g),
                                     buf, len(buf)))
    else:
        ql = np.ascontiguousarray(labels, dtype=np.uint32)
        _need_host(ql, k, "labels")
        ls = np.ascontiguousarray([] if lstart is None else lstart, dtype=np.uint32)
        if len(ls) < 2:
            raise HugeError(EINVAL, "lstart needs nlabels + 1 >= 2 entries")
        _check(lib.huge_plan_offline_labeled(k, _ptr(e), len(edges), _ptr(ql), _ptr(ls), len(ls) - 1, _ptr(o),
                                             _ptr(pa), npo, flags, _ptr(c), float(edges_g), buf, len(buf)))
    return json.loads(buf.value.decode())


def enumerate(plan: Plan, mode: int = COUNT, mem_bound: int = 1 << 30, sink=None, stream=None,
              roots=None, root_range=None, flags: int = 0, level_cap: int = 0, chunk_roots: int = 0,
              root_weights=None, drain=None, stats: bool = False, time_limit_ms: int = 0,
              variant: int = 0):
    """huge_enumerate_ex. sink: a CUDA uint32 tensor of shape (rows, k) for LIST mode; drain:
    optional callable(ptr:int, nrows:int) called when it is full. Returns the count, or
    (count, stats dict) with stats=True."""
    lib = load()
    o = EnumOpts()
    keep = []
    if roots is not None:
        r = np.ascontiguousarray(roots, dtype=np.uint32)
        keep.append(r)
        o.roots, o.nroots = r.ctypes.data, len(r)
    if root_range is not None:
        o.root_begin, o.root_end = root_range
    if root_weights is not None:
        w = np.ascontiguousarray(root_weights, dtype=np.float32)
        _need_host(w, plan.graph.info()["n"], "root_weights")
        keep.append(w)
        o.root_weights = w.ctypes.data
    o.flags, o.level_cap, o.chunk_roots = flags, level_cap, chunk_roots
    o.time_limit_ms = time_limit_ms
    o.variant = variant
    sk = None
    if sink is not None:
        _need_device(sink, 0, "sink", dtypes=("int32", "uint32"), width=plan.k)  # rows of k ids
        sk = Sink()
        sk.rows = _ptr(sink).value
        sk.capacity_rows = sink.shape[0]
        if drain is not None:
            cb = DRAIN_FN(lambda ctx, rows, n: drain(rows, n))
            keep.append(cb)
            sk.drain = cb
        else:
            sk.drain = DRAIN_FN()
    cnt = ctypes.c_int64()
    st = Stats()
    _check(lib.huge_enumerate_ex(plan.handle, mode, mem_bound, ctypes.byref(sk) if sk else None,
                                 _stream_ptr(stream), ctypes.byref(o), ctypes.byref(cnt), ctypes.byref(st)))
    return (cnt.value, st.as_dict()) if stats else cnt.value


def enumerate_batch(plans, mem_bound: int = 1 << 30, stream=None, stats: bool = False, roots=None,
                    level_caps=None, variants=None, flags: int = 0, time_limit_ms: int = 0, level_rows=None):
    """huge_enumerate_batch_ex: one persistent launch for all plans. roots: None, or one root
    array (or None) per plan; level_caps / variants: None or one value per plan; level_rows: an
    optional int64 array of shape (len(plans), 16) that receives each plan's rows per level."""
    lib = load()
    nq = len(plans)
    arr = (ctypes.c_void_p * nq)(*[p.handle.value for p in plans])
    out = np.zeros(nq, dtype=np.int64)
    st = Stats()
    opts = (EnumOpts * nq)()
    keep = []
    for i in range(nq):
        o = opts[i]
        if roots is not None and roots[i] is not None:
            r = np.ascontiguousarray(roots[i], dtype=np.uint32)
            keep.append(r)
            o.roots, o.nroots = r.ctypes.data, len(r)
            if len(r) == 0:
                o.roots, o.nroots = None, 0
                o.root_begin, o.root_end = 1, 1  # an empty range: no tasks for this plan
        if level_caps is not None:
            o.level_cap = int(level_caps[i])
        if variants is not None:
            o.variant = int(variants[i])
        o.flags, o.time_limit_ms = flags, time_limit_ms
    lr = None
    if level_rows is not None:
        if level_rows.dtype != np.int64 or level_rows.shape != (nq, 16) or not level_rows.flags.c_contiguous:
            raise ValueError("level_rows must be a C-contiguous int64 array of shape (len(plans), 16)")
        lr = level_rows
    _check(lib.huge_enumerate_batch_ex(arr, nq, mem_bound, _stream_ptr(stream), ctypes.cast(opts, ctypes.c_void_p),
                                       _ptr(out), _ptr(lr), ctypes.byref(st)))
    return (out, st.as_dict()) if stats else out


def autotune(plans, mem_bound: int = 1 << 30, budget_ms: float = 2000.0, stream=None):
    lib = load()
    arr = (ctypes.c_void_p * len(plans))(*[p.handle.value for p in plans])
    cap, chunk = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib.huge_autotune(arr, len(plans), mem_bound, budget_ms, _stream_ptr(stream), ctypes.byref(cap),
                             ctypes.byref(chunk)))
    return cap.value, chunk.value


def count_noalloc(d_offsets, d_adj, n: int, nnz: int, k: int, edges, order=None, po=None, stream=None) -> int:
    """huge_count_noalloc: COUNT on a CSR already on the device (uint32 offsets and adjacency,
    as device pointers or CUDA tensors), using only the library's static scratch. The C side
    reads the arrays as given, so tensors are checked here first: contiguous, a 4-byte integer
    dtype, on the current CUDA device, with at least n + 1 offsets and nnz adjacency entries."""
    lib = load()
    for name, t, need in (("d_offsets", d_offsets, n + 1), ("d_adj", d_adj, nnz)):
        _need_device(t, need, name, dtypes=("int32", "uint32"))
    e = np.asarray([x for uv in edges for x in uv] or [0], dtype=np.uint32)
    o = None if order is None else np.asarray(order, dtype=np.uint32)
    _need_host(o, k, "order")
    if po is None:
        pa, npo = None, -1
    else:
        pa = np.asarray([x for ab in po for x in ab] or [0], dtype=np.uint32)
        npo = len(po)
    cnt = ctypes.c_int64()
    _check(lib.huge_count_noalloc(_ptr(d_offsets), _ptr(d_adj), n, nnz, k, _ptr(e), len(edges), _ptr(o), _ptr(pa),
                                  npo, _stream_ptr(stream), ctypes.byref(cnt)))
    return cnt.value


class MLP:
    """The learned cardinality estimator (huge_mlp_*). Tensors are CUDA float32 torch tensors."""

    def __init__(self, seed: int = 0):
        h = ctypes.c_void_p()
        _check(load().huge_mlp_create(seed, ctypes.byref(h)))
        self.handle = h
        self.n_params = load().huge_mlp_num_params()

    def set_params(self, params=None, mu=None, sd=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32).ravel() for a in (params, mu, sd)]
        for a, need, name in zip(arrs, (self.n_params, 64, 64), ("params", "mu", "sd")):
            _need_host(a, need, name)
        _check(load().huge_mlp_set_params(self.handle, *[_ptr(a) for a in arrs]))

    def get_params(self):
        p = np.zeros(self.n_params, np.float32)
        mu = np.zeros(64, np.float32)
        sd = np.zeros(64, np.float32)
        _check(load().huge_mlp_get_params(self.handle, _ptr(p), _ptr(mu), _ptr(sd)))
        return p, mu, sd

    def forward(self, x, y, stream=None):
        _need_device(x, 0, "x", width=64)
        _need_device(y, x.shape[0], "y")
        _check(load().huge_mlp_forward(self.handle, _ptr(x), x.shape[0], _ptr(y), _stream_ptr(stream)))

    def loss_grad(self, x, t, grad, stream=None):
        _need_device(x, 0, "x", width=64)
        _need_device(t, x.shape[0], "t")
        _need_device(grad, self.n_params, "grad")
        loss = ctypes.c_float()
        _check(load().huge_mlp_loss_grad(self.handle, _ptr(x), _ptr(t), x.shape[0], _ptr(grad), ctypes.byref(loss),
                                         _stream_ptr(stream)))
        return loss.value

    def train(self, x, t, epochs: int, batch_rows: int = 8192, lr: float = 1e-3, stream=None):
        _need_device(x, 0, "x", width=64)
        _need_device(t, x.shape[0], "t")
        loss = ctypes.c_float()
        _check(load().huge_mlp_train(self.handle, _ptr(x), _ptr(t), x.shape[0], epochs, batch_rows, lr,
                                     ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value

    def free(self):
        if self.handle:
            load().huge_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def root_features(plan: Plan, roots) -> np.ndarray:
    """huge_root_features: (len(roots), 64) float32 features of (plan, root) pairs."""
    r = np.ascontiguousarray(roots, dtype=np.uint32)
    out = np.zeros((max(len(r), 1), 64), np.float32)
    _check(load().huge_root_features(plan.handle, _ptr(r), len(r), _ptr(out)))
    return out[: len(r)]


def plan_features(graph: Graph, k: int, edges, mask: int, po=None) -> np.ndarray:
    e = np.asarray([x for uv in edges for x in uv] or [0], dtype=np.uint32)
    if po is None:
        pa, npo = None, -1
    else:
        pa = np.asarray([x for ab in po for x in ab] or [0], dtype=np.uint32)
        npo = len(po)
    out = np.zeros(64, np.float32)
    _check(load().huge_plan_features(graph.handle, k, _ptr(e), len(edges), _ptr(pa), npo, mask, _ptr(out)))
    return out
