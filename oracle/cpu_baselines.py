"""CPU baselines for bench.py's cpu_baseline leg — NOT the oracle.

Thin ctypes wrappers of ``cpu_baselines.c`` (OpenMP pull supersteps on all
host cores, a binary-heap Dijkstra and a union-find on one core). They are
timed beside the GPU numbers; no parity check of the CUDA path uses them.
The input preparation (CSC / CSR construction) is done here in numpy and is
not part of what the bench times.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "cpu_baselines.c")
_LIB = os.path.join(_DIR, "_build", "libcpubase.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_SRC) > os.path.getmtime(_LIB):
        cc = shutil.which("gcc") or "cc"
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_LIB))
        os.close(fd)
        try:
            p = subprocess.run([cc, "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp],
                               stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
            if p.returncode != 0:
                raise RuntimeError("cpu baseline build failed:\n" + p.stdout)
            os.replace(tmp, _LIB)
        finally:
            if os.path.exists(tmp):
                os.unlink(tmp)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        u64, u32, i64, dbl, p = C.c_uint64, C.c_uint32, C.c_int64, C.c_double, C.c_void_p
        lib.cb_threads.restype = C.c_int
        lib.cb_set_threads.argtypes = [C.c_int]
        lib.cb_pagerank_pull.restype = C.c_int
        lib.cb_pagerank_pull.argtypes = [u64, p, p, p, dbl, u32, p]
        lib.cb_minlabel_pull.restype = i64
        lib.cb_minlabel_pull.argtypes = [u64, p, p, p, p, u32]
        lib.cb_dijkstra.restype = C.c_int
        lib.cb_dijkstra.argtypes = [u64, p, p, p, u32, p]
        lib.cb_union_find.argtypes = [u64, u64, p, p, p]
        lib.cb_csc_build.restype = C.c_int
        lib.cb_csc_build.argtypes = [u64, u64, p, p, p, p, p, p]
        _lib = lib
    return _lib


def host_cores() -> int:
    """Cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def set_threads(t: int) -> int:
    lib = _load()
    lib.cb_set_threads(int(t))
    return int(lib.cb_threads())


def _p(a):
    return a.ctypes.data


def csc(n, src, dst, w=None):
    """(col_ptr u64[n+1], sources, weights or None) grouped by destination
    (a stable counting sort in C)."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    col_ptr = np.empty(n + 1, np.uint64)
    s = np.empty(max(len(src), 1), np.uint32)
    ws = None
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.uint32)
        ws = np.empty(max(len(src), 1), np.uint32)
    if _load().cb_csc_build(n, len(src), _p(src), _p(dst), None if w is None else _p(w), _p(col_ptr), _p(s),
                            None if ws is None else _p(ws)):
        raise MemoryError("cpu baseline allocation failed")
    return col_ptr, s[:len(src)], None if ws is None else ws[:len(src)]


def csr(n, src, dst, w):
    order = np.argsort(src, kind="stable")
    row_ptr = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    return row_ptr, np.ascontiguousarray(dst[order], dtype=np.uint32), np.ascontiguousarray(w[order], dtype=np.uint32)


def pagerank_pull(n, col_ptr, csrc, outdeg, damping, iters):
    r = np.empty(n, np.float64)
    od = np.ascontiguousarray(outdeg, dtype=np.uint32)
    if _load().cb_pagerank_pull(n, _p(col_ptr), _p(csrc), _p(od), damping, iters, _p(r)):
        raise MemoryError("cpu baseline allocation failed")
    return r


def minlabel_pull(n, col_ptr, csrc, cw, x0, max_steps=1 << 30):
    x = np.ascontiguousarray(x0, dtype=np.uint32).copy()
    steps = _load().cb_minlabel_pull(n, _p(col_ptr), _p(csrc), None if cw is None else _p(cw), _p(x),
                                     min(max_steps, n + 2))
    if steps < 0:
        raise MemoryError("cpu baseline allocation failed")
    return x, int(steps)


def dijkstra(n, row_ptr, cdst, cw, source):
    d = np.empty(n, np.uint32)
    if _load().cb_dijkstra(n, _p(row_ptr), _p(cdst), _p(cw), source, _p(d)):
        raise MemoryError("cpu baseline allocation failed")
    return d


def union_find(n, src, dst):
    lab = np.empty(n, np.uint32)
    s = np.ascontiguousarray(src, dtype=np.uint32)
    t = np.ascontiguousarray(dst, dtype=np.uint32)
    _load().cb_union_find(n, len(s), _p(s), _p(t), _p(lab))
    return lab
