"""ctypes binding of libgxp.so (the C-ABI in ``include/gxp.h``).

Argument marshalling only: every step of the superstep path runs in the
library's CUDA kernels. The raw functions keep the C names (``gxp_init``,
``gxp_load_partition``, ``gxp_superstep``, ``gxp_sync`` ...); ``Context`` is a
thin convenience wrapper that turns status codes into exceptions and accepts
numpy arrays (host) or CUDA tensors (device) through their data pointers.

Loading fails loudly when the library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

# status codes
GXP_OK, GXP_E_INVAL, GXP_E_NOMEM, GXP_E_CUDA, GXP_E_TIMEOUT = 0, 1, 2, 3, 4
GXP_E_BOUNDS, GXP_E_STATE, GXP_E_UNSUPPORTED, GXP_E_BUSY, GXP_E_LOST = 5, 6, 7, 8, 9
# host-side fault injection (gxp_config.fault)
GXP_FAULT_NONE, GXP_FAULT_ALLOC, GXP_FAULT_H2D, GXP_FAULT_SYNC_DROP, GXP_FAULT_TIMEOUT = 0, 1, 2, 3, 4
# algorithms and template operators
GXP_ALGO_SSSP, GXP_ALGO_CC, GXP_ALGO_PAGERANK, GXP_ALGO_PPR, GXP_ALGO_LP = 0, 1, 2, 3, 4
GXP_GEN_RELAX, GXP_GEN_LABEL, GXP_GEN_CONTRIB = 0, 1, 2
GXP_MERGE_MIN, GXP_MERGE_SUM, GXP_MERGE_MODE = 0, 1, 2
GXP_APPLY_MIN, GXP_APPLY_PAGERANK, GXP_APPLY_SET = 0, 1, 2
GXP_FMT_COO, GXP_FMT_CSC, GXP_FMT_CSR = 0, 1, 2
ALL_PARTS = 0xFFFFFFFF
INF = 0xFFFFFFFF

TEMPLATES = {
    GXP_ALGO_SSSP: (GXP_GEN_RELAX, GXP_MERGE_MIN, GXP_APPLY_MIN),
    GXP_ALGO_CC: (GXP_GEN_LABEL, GXP_MERGE_MIN, GXP_APPLY_MIN),
    GXP_ALGO_PAGERANK: (GXP_GEN_CONTRIB, GXP_MERGE_SUM, GXP_APPLY_PAGERANK),
    GXP_ALGO_PPR: (GXP_GEN_CONTRIB, GXP_MERGE_SUM, GXP_APPLY_PAGERANK),
    GXP_ALGO_LP: (GXP_GEN_LABEL, GXP_MERGE_MODE, GXP_APPLY_SET),
}
# serving
GXP_QUERY_SSSP, GXP_QUERY_PPR = 0, 1
GXP_QUERY_QUEUED, GXP_QUERY_RUNNING, GXP_QUERY_DONE, GXP_QUERY_FAILED = 0, 1, 2, 3
GXP_DIR_AUTO, GXP_DIR_PULL, GXP_DIR_PUSH = 0, 1, 2
GXP_CACHE_NONE = 0xFFFFFFFF


class gxp_config(C.Structure):
    _fields_ = [("mem_budget", C.c_uint64), ("tile_items", C.c_uint32), ("hub_items", C.c_uint32),
                ("timeout_ns", C.c_uint64), ("check_bounds", C.c_uint32), ("max_slots", C.c_uint32),
                ("pipeline_depth", C.c_uint32), ("keep_ids", C.c_uint32), ("direction", C.c_uint32),
                ("push_div", C.c_uint32), ("cache_slots", C.c_uint32), ("fault", C.c_uint32),
                ("fault_at", C.c_uint32), ("reserved", C.c_uint32 * 1)]


class gxp_stats(C.Structure):
    _fields_ = [("supersteps", C.c_uint64), ("edges_scanned", C.c_uint64), ("last_changed", C.c_uint64),
                ("last_boundary_changed", C.c_uint64), ("syncs_done", C.c_uint64),
                ("syncs_skipped", C.c_uint64), ("sync_pairs", C.c_uint64), ("last_l1_delta", C.c_double),
                ("last_dangling", C.c_double), ("last_superstep_ms", C.c_double),
                ("device_bytes", C.c_uint64), ("push_supersteps", C.c_uint64), ("cache_downloads", C.c_uint64),
                ("last_kernel_ms", C.c_double), ("persistent_launches", C.c_uint64),
                ("reserved", C.c_uint64 * 2)]


# (name, restype, argtypes) of every exported symbol
_P, _U32, _U64, _I, _F, _D = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int, C.c_float, C.c_double
SIGNATURES = [
    ("gxp_config_default", None, [_P]),
    ("gxp_init", _I, [_I, _P, _P]),
    ("gxp_destroy", None, [_P]),
    ("gxp_status_string", C.c_char_p, [_I]),
    ("gxp_last_error", C.c_char_p, [_P]),
    ("gxp_set_stream", _I, [_P, _P]),
    ("gxp_create_graph", _I, [_P, _U64, _U32, _P]),
    ("gxp_load_partition", _I, [_P, _U32, _I, _U64, _P, _P, _P]),
    ("gxp_begin", _I, [_P, _I, _U32, _F]),
    ("gxp_get_values", _I, [_P, _U32, _P, _U64]),
    ("gxp_set_values", _I, [_P, _U32, _P, _U64]),
    ("gxp_superstep", _I, [_P, _I, _I, _I, _I, _P]),
    ("gxp_sync", _I, [_P, _U32, _P, _P, _U64, _P, _P]),
    ("gxp_run", _I, [_P, _I, _U32, _F, _U32, _P]),
    ("gxp_cache_get", _I, [_P, _U32, _P, _U64, _P]),
    ("gxp_tune_cache_get", _I, [C.c_char_p, C.c_char_p, _P]),
    ("gxp_tune_cache_put", _I, [C.c_char_p, C.c_char_p, _P]),
    ("gxp_stats_get", _I, [_P, _P]),
    ("gxp_block_size_model", _I, [_D, _D, _D, _D, _U64, _P, _P, _P]),
    ("gxp_superstep_min_noalloc", _I, [_I, _U32, _U64, _P, _P, _P, _P, _P, _P, _P]),
    ("gxp_sssp_batch", _I, [_P, _P, _U32, _P, _P, _P]),
    ("gxp_serve_add_graph", _I, [_P, _U64, _U64, _P, _P, _P, _P]),
    ("gxp_serve_start", _I, [_P, _P]),
    ("gxp_serve_stop", _I, [_P]),
    ("gxp_query_submit", _I, [_P, _U32, _I, _U32, _F, _U32, _P]),
    ("gxp_query_poll", _I, [_P, _U64, _P, _U64, _I, _P]),
    ("gxp_query_next_done", _I, [_P, _I, _P]),
    ("gxp_query_info_get", _I, [_P, _U64, _P]),
    ("gxp_serve_report_get", _I, [_P, _P]),
]

_lib = None


def lib_path() -> str:
    return _build.GXP_LIB


def load(build_if_missing: bool = True):
    """Load libgxp.so (building it first if asked); raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build_gxp()
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libgxp.so not found at {path}: run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GxpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_status_name(code)}: {msg}")
        self.code = code


def _status_name(code: int) -> str:
    return load().gxp_status_string(code).decode()


def _ptr(x):
    """Data pointer of a numpy array, a torch tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)!r}")


def block_size_model(k1: float, k2: float, k3: float, a: float, d: int):
    """Lemma 1 with the integer rounding step: returns (b, s, t_estimate)."""
    b, s, t = C.c_uint64(), C.c_uint64(), C.c_double()
    rc = load().gxp_block_size_model(k1, k2, k3, a, d, C.byref(b), C.byref(s), C.byref(t))
    if rc:
        raise GxpError(rc, load().gxp_last_error(None).decode())
    return b.value, s.value, t.value


class gxp_batch_opts(C.Structure):
    _fields_ = [("streamed", C.c_uint32), ("pipelined", C.c_uint32), ("block_edges", C.c_uint64),
                ("use_graph", C.c_uint32), ("max_steps", C.c_uint32), ("tune_cache", C.c_char_p),
                ("reserved", C.c_uint32 * 4)]


class gxp_batch_report(C.Structure):
    _fields_ = [("supersteps", C.c_uint32), ("blocks", C.c_uint32), ("block_edges", C.c_uint64),
                ("ms_total", C.c_double), ("k1", C.c_double), ("k2", C.c_double), ("k3", C.c_double),
                ("a", C.c_double), ("model_block_edges", C.c_double), ("model_ms", C.c_double),
                ("sweep_best_ms", C.c_double), ("edges_per_superstep", C.c_uint64),
                ("tune_from_cache", C.c_uint64), ("active_edges", C.c_uint64), ("persistent", C.c_uint64),
                ("reserved", C.c_uint64 * 3)]


class gxp_tune_record(C.Structure):
    _fields_ = [("k1", C.c_double), ("k2", C.c_double), ("k3", C.c_double), ("a", C.c_double),
                ("model_block_edges", C.c_double), ("block_edges", C.c_double), ("sweep_best_ms", C.c_double)]


class Context:
    """One gxp_ctx: a device, a partitioned graph and a running algorithm."""

    def __init__(self, device: int = 0, tile_items: int = 0, hub_items: int = 0,
                 check_bounds: bool = False, timeout_ns: int = 0, mem_budget: int = 0, keep_ids: bool = False,
                 direction: int = GXP_DIR_AUTO, push_div: int = 0, cache_slots: int = 0,
                 fault: int = GXP_FAULT_NONE, fault_at: int = 0):
        self.lib = load()
        cfg = gxp_config()
        self.lib.gxp_config_default(C.byref(cfg))
        cfg.fault, cfg.fault_at = fault, fault_at
        cfg.tile_items, cfg.hub_items, cfg.keep_ids = tile_items, hub_items, int(keep_ids)
        cfg.direction, cfg.push_div, cfg.cache_slots = direction, push_div, cache_slots
        cfg.check_bounds, cfg.timeout_ns, cfg.mem_budget = int(check_bounds), timeout_ns, mem_budget
        h = C.c_void_p()
        rc = self.lib.gxp_init(device, C.byref(cfg), C.byref(h))
        if rc:
            raise GxpError(rc, self.lib.gxp_last_error(None).decode())
        self.h = h
        self.n_vertices = 0
        self.n_parts = 0
        self.bounds = None
        self.algo = None

    def _ck(self, rc: int):
        if rc:
            raise GxpError(rc, self.lib.gxp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.gxp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ----------------------------------------------------------------- graph
    def set_stream(self, stream):
        self._ck(self.lib.gxp_set_stream(self.h, stream))

    def create_graph(self, n_vertices: int, n_parts: int = 1, part_begin=None):
        pb = None
        if part_begin is not None:
            pb = np.ascontiguousarray(part_begin, dtype=np.uint64)
        self._ck(self.lib.gxp_create_graph(self.h, n_vertices, n_parts, _ptr(pb)))
        self.n_vertices, self.n_parts = n_vertices, n_parts
        self.bounds = (pb.tolist() if pb is not None
                       else [n_vertices * p // n_parts for p in range(n_parts + 1)])

    def load_partition(self, part: int, fmt: int, n_edges: int, idx0, idx1, weights=None):
        self._ck(self.lib.gxp_load_partition(self.h, part, fmt, n_edges, _ptr(idx0), _ptr(idx1),
                                             _ptr(weights)))

    def load_coo(self, src, dst, w=None):
        """Split a whole-graph COO list by destination owner and load every partition."""
        src = np.ascontiguousarray(src, dtype=np.uint32)
        dst = np.ascontiguousarray(dst, dtype=np.uint32)
        w = None if w is None else np.ascontiguousarray(w, dtype=np.uint32)
        if self.n_parts == 1:
            self.load_partition(0, GXP_FMT_COO, len(src), src, dst, w)
            return
        b = np.asarray(self.bounds, dtype=np.int64)
        owner = np.searchsorted(b, dst, side="right") - 1
        order = np.argsort(owner, kind="stable")
        cuts = np.searchsorted(owner[order], np.arange(self.n_parts + 1))
        for p in range(self.n_parts):
            sel = order[cuts[p]:cuts[p + 1]]
            ws = None if w is None else np.ascontiguousarray(w[sel])
            self.load_partition(p, GXP_FMT_COO, len(sel), np.ascontiguousarray(src[sel]),
                                np.ascontiguousarray(dst[sel]), ws)

    # ------------------------------------------------------------- algorithm
    def begin(self, algo: int, source: int = 0, damping: float = 0.85):
        self._ck(self.lib.gxp_begin(self.h, algo, source, damping))
        self.algo = algo

    def superstep(self, algo=None, template=None, want_changed: bool = True):
        algo = self.algo if algo is None else algo
        g, m, a = template if template is not None else TEMPLATES[algo]
        n = C.c_uint64()
        self._ck(self.lib.gxp_superstep(self.h, algo, g, m, a, C.byref(n) if want_changed else None))
        return n.value if want_changed else None

    def run(self, algo: int, source: int = 0, damping: float = 0.85, max_steps: int = 1 << 30) -> int:
        s = C.c_uint32()
        self._ck(self.lib.gxp_run(self.h, algo, source, damping, max_steps, C.byref(s)))
        self.algo = algo
        return s.value

    def values(self, part: int = ALL_PARTS, out=None):
        n = self.n_vertices if part == ALL_PARTS else int(self.bounds[part + 1] - self.bounds[part])
        if out is None:
            out = np.empty(n, dtype=np.float32 if self.algo in (GXP_ALGO_PAGERANK, GXP_ALGO_PPR) else np.uint32)
        self._ck(self.lib.gxp_get_values(self.h, part, _ptr(out), n))
        return out

    def set_values(self, arr, part: int = ALL_PARTS):
        arr = np.ascontiguousarray(arr)
        self._ck(self.lib.gxp_set_values(self.h, part, _ptr(arr), len(arr)))

    def cache(self, part: int) -> np.ndarray:
        """Vertex ids of the copies partition `part` holds cached now (ascending)."""
        n = C.c_uint64()
        rc = self.lib.gxp_cache_get(self.h, part, None, 0, C.byref(n))
        if rc not in (GXP_OK, GXP_E_INVAL) or (rc == GXP_E_INVAL and n.value == 0):
            self._ck(rc)
        out = np.empty(max(n.value, 1), dtype=np.uint32)
        self._ck(self.lib.gxp_cache_get(self.h, part, _ptr(out), n.value, C.byref(n)))
        return out[:n.value]

    def sync(self, part: int):
        """(ids, values, skipped) of partition `part`'s last upload (Algorithm 3)."""
        n, sk = C.c_uint64(), C.c_int()
        rc = self.lib.gxp_sync(self.h, part, None, None, 0, C.byref(n), C.byref(sk))
        if rc not in (GXP_OK, GXP_E_INVAL):
            self._ck(rc)
        cnt = n.value
        ids = np.empty(max(cnt, 1), dtype=np.uint32)
        vals = np.empty(max(cnt, 1), dtype=np.float32 if self.algo in (GXP_ALGO_PAGERANK, GXP_ALGO_PPR)
                        else np.uint32)
        self._ck(self.lib.gxp_sync(self.h, part, _ptr(ids), _ptr(vals), cnt, C.byref(n), C.byref(sk)))
        return ids[:cnt], vals[:cnt], bool(sk.value)

    def sssp_batch(self, sources, out=None, streamed=False, pipelined=True, block_edges=0,
                   use_graph=False, max_steps=0, tune_cache=None):
        """Multi-source SSSP: returns (dist uint32[V][n_sources] (or `out`), report dict)."""
        srcs = np.ascontiguousarray(sources, dtype=np.uint32)
        if out is None:
            out = np.empty((self.n_vertices, len(srcs)), dtype=np.uint32)
        o = gxp_batch_opts()
        o.streamed, o.pipelined, o.block_edges = int(streamed), int(pipelined), block_edges
        o.use_graph, o.max_steps = int(use_graph), max_steps
        o.tune_cache = None if tune_cache is None else os.fsencode(tune_cache)
        r = gxp_batch_report()
        self._ck(self.lib.gxp_sssp_batch(self.h, _ptr(srcs), len(srcs), _ptr(out), C.byref(o), C.byref(r)))
        return out, {k: getattr(r, k) for k, _ in gxp_batch_report._fields_ if k != "reserved"}

    def stats(self) -> dict:
        s = gxp_stats()
        self._ck(self.lib.gxp_stats_get(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in gxp_stats._fields_ if k != "reserved"}


class gxp_serve_opts(C.Structure):
    _fields_ = [("max_slots", C.c_uint32), ("results_per_graph", C.c_uint32), ("queue_cap", C.c_uint32),
                ("priorities", C.c_uint32), ("reserved", C.c_uint32 * 8)]


class gxp_query_info(C.Structure):
    _fields_ = [("state", C.c_uint32), ("supersteps", C.c_uint32), ("graph", C.c_uint32), ("kind", C.c_uint32),
                ("n_values", C.c_uint64), ("queue_ms", C.c_double), ("run_ms", C.c_double),
                ("reserved", C.c_uint64 * 4)]


class gxp_serve_report(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("queued", C.c_uint64), ("running", C.c_uint64), ("sssp_supersteps", C.c_uint64),
                ("ppr_supersteps", C.c_uint64), ("device_bytes", C.c_uint64), ("reserved", C.c_uint64 * 8)]


class Server:
    """Query server of one context (gxp_serve_* / gxp_query_*): graphs made
    resident, then SSSP / personalized-PageRank queries served by continuous
    batching. The query methods may be called from several threads."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        self.lib = ctx.lib
        self.n = []   # vertices per graph

    def _ck(self, rc: int):
        if rc:
            raise GxpError(rc, self.lib.gxp_last_error(None).decode())

    def add_graph(self, n_vertices: int, src, dst, w=None) -> int:
        src = src if hasattr(src, "data_ptr") else np.ascontiguousarray(src, dtype=np.uint32)
        dst = dst if hasattr(dst, "data_ptr") else np.ascontiguousarray(dst, dtype=np.uint32)
        if w is not None and not hasattr(w, "data_ptr"):
            w = np.ascontiguousarray(w, dtype=np.uint32)
        g = C.c_uint32()
        self._ck(self.lib.gxp_serve_add_graph(self.ctx.h, n_vertices, len(src), _ptr(src), _ptr(dst), _ptr(w),
                                              C.byref(g)))
        self.n.append(n_vertices)
        return g.value

    def start(self, max_slots: int = 0, results_per_graph: int = 0, queue_cap: int = 0, priorities: bool = False):
        o = gxp_serve_opts()
        o.max_slots, o.results_per_graph, o.queue_cap = max_slots, results_per_graph, queue_cap
        o.priorities = int(priorities)
        self._ck(self.lib.gxp_serve_start(self.ctx.h, C.byref(o)))

    def stop(self):
        self._ck(self.lib.gxp_serve_stop(self.ctx.h))

    def submit(self, graph: int, kind: int, source: int, damping: float = 0.85, iters: int = 0) -> int:
        q = C.c_uint64()
        self._ck(self.lib.gxp_query_submit(self.ctx.h, graph, kind, source, damping, iters, C.byref(q)))
        return q.value

    def poll(self, qid: int, out=None, timeout_ms: int = -1) -> bool:
        """Wait for qid; with `out` (numpy or tensor of >= n_vertices 4-byte
        values) copy the result there and release the query. Returns done."""
        d = C.c_int()
        cap = 0 if out is None else (out.numel() if hasattr(out, "numel") else out.size)
        self._ck(self.lib.gxp_query_poll(self.ctx.h, qid, _ptr(out), cap, timeout_ms, C.byref(d)))
        return bool(d.value)

    def result(self, qid: int, kind: int, graph: int):
        """Blocking: the result of qid as a new numpy array (uint32 or float32)."""
        out = np.empty(self.n[graph], dtype=np.uint32 if kind == GXP_QUERY_SSSP else np.float32)
        self.poll(qid, out, -1)
        return out

    def next_done(self, timeout_ms: int = -1) -> int:
        q = C.c_uint64()
        self._ck(self.lib.gxp_query_next_done(self.ctx.h, timeout_ms, C.byref(q)))
        return q.value

    def info(self, qid: int) -> dict:
        i = gxp_query_info()
        self._ck(self.lib.gxp_query_info_get(self.ctx.h, qid, C.byref(i)))
        return {k: getattr(i, k) for k, _ in gxp_query_info._fields_ if k != "reserved"}

    def report(self) -> dict:
        r = gxp_serve_report()
        self._ck(self.lib.gxp_serve_report_get(self.ctx.h, C.byref(r)))
        return {k: getattr(r, k) for k, _ in gxp_serve_report._fields_ if k != "reserved"}
