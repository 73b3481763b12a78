"""CPU oracle for the GAS superstep engine — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package. It shares no
code with the CUDA path: ``oracle.c`` is plain single-threaded C (fp64 for
PageRank), ``lemma1.py`` restates Lemma 1 and the pipeline-time equation of
Section III-A, and ``sync.py`` states the lazy-uploading and skipping rules of
Section III-B in numpy.

Pins (what holds this oracle to something other than itself) live in
``tests/test_oracle_pins.py``: SciPy's Dijkstra and connected components,
hand-built graphs, closed forms for PageRank and for mode-label propagation
on cliques, stars, paths and oscillating pairs, dense linear solves, and
brute force for Lemma 1.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "oracle.c")
_LIB = os.path.join(_DIR, "_build", "liboracle.so")
INF = 0xFFFFFFFF

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no OpenMP: the oracle is single-threaded)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_SRC) > os.path.getmtime(_LIB):
        cc = shutil.which("gcc") or "cc"
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_LIB))
        os.close(fd)
        try:
            p = subprocess.run([cc, "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"],
                               stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
            if p.returncode != 0:
                raise RuntimeError("oracle build failed:\n" + p.stdout)
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
        lib.orc_sssp_step.restype = u64
        lib.orc_sssp_step.argtypes = [u64, u64, p, p, p, p, p, p]
        lib.orc_sssp.restype = i64
        lib.orc_sssp.argtypes = [u64, u64, p, p, p, u32, u32, p, p]
        lib.orc_cc_step.restype = u64
        lib.orc_cc_step.argtypes = [u64, u64, p, p, p, p, p]
        lib.orc_cc.restype = i64
        lib.orc_cc.argtypes = [u64, u64, p, p, u32, p, p]
        lib.orc_lp_step.restype = u64
        lib.orc_lp_step.argtypes = [u64, u64, p, p, p, p, p]
        lib.orc_lp.restype = i64
        lib.orc_lp.argtypes = [u64, u64, p, p, u32, p, p]
        lib.orc_pr_step.restype = dbl
        lib.orc_pr_step.argtypes = [u64, u64, p, p, p, dbl, p, p, p]
        lib.orc_pagerank.restype = C.c_int
        lib.orc_pagerank.argtypes = [u64, u64, p, p, dbl, u32, p, p, p]
        lib.orc_ppr.restype = C.c_int
        lib.orc_ppr.argtypes = [u64, u64, p, p, u32, dbl, u32, p]
        lib.orc_outdeg.argtypes = [u64, u64, p, p]
        _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def sssp(n, src, dst, w, source, max_steps=1 << 30):
    """Jacobi Bellman-Ford to convergence. Returns (dist u32[n], supersteps, changed[])."""
    src, dst, w = _u32(src), _u32(dst), _u32(w)
    dist = np.empty(n, dtype=np.uint32)
    cap = min(max_steps, n + 2)
    changed = np.zeros(cap, dtype=np.uint64)
    steps = _load().orc_sssp(n, len(src), _p(src), _p(dst), _p(w), source, cap,
                             _p(dist), _p(changed))
    if steps < 0:
        raise MemoryError("oracle sssp allocation failed")
    return dist, int(steps), changed[:steps].copy()


def sssp_step(n, src, dst, w, d_in):
    src, dst, w, d_in = _u32(src), _u32(dst), _u32(w), _u32(d_in)
    d_out = np.empty(n, dtype=np.uint32)
    msg = np.empty(n, dtype=np.uint64)
    c = _load().orc_sssp_step(n, len(src), _p(src), _p(dst), _p(w), _p(d_in), _p(d_out), _p(msg))
    return d_out, int(c)


def cc(n, src, dst, max_steps=1 << 30):
    """Min-label propagation to convergence. Returns (labels u32[n], supersteps, changed[])."""
    src, dst = _u32(src), _u32(dst)
    labels = np.empty(n, dtype=np.uint32)
    cap = min(max_steps, n + 2)
    changed = np.zeros(cap, dtype=np.uint64)
    steps = _load().orc_cc(n, len(src), _p(src), _p(dst), cap, _p(labels), _p(changed))
    if steps < 0:
        raise MemoryError("oracle cc allocation failed")
    return labels, int(steps), changed[:steps].copy()


def cc_step(n, src, dst, l_in):
    src, dst, l_in = _u32(src), _u32(dst), _u32(l_in)
    l_out = np.empty(n, dtype=np.uint32)
    msg = np.empty(n, dtype=np.uint32)
    c = _load().orc_cc_step(n, len(src), _p(src), _p(dst), _p(l_in), _p(l_out), _p(msg))
    return l_out, int(c)


LP_MAX_STEPS = 15   # Section V-A caps LP at 15 iterations


def lp(n, src, dst, max_steps=LP_MAX_STEPS):
    """Synchronous mode-label propagation from l_0[v] = v until a superstep
    changes nothing or max_steps. Returns (labels u32[n], supersteps, changed[])."""
    src, dst = _u32(src), _u32(dst)
    labels = np.empty(n, dtype=np.uint32)
    cap = max(1, max_steps)
    changed = np.zeros(cap, dtype=np.uint64)
    steps = _load().orc_lp(n, len(src), _p(src), _p(dst), max_steps, _p(labels), _p(changed))
    if steps < 0:
        raise MemoryError("oracle lp allocation failed")
    return labels, int(steps), changed[:steps].copy()


def lp_step(n, src, dst, l_in):
    src, dst, l_in = _u32(src), _u32(dst), _u32(l_in)
    l_out = np.empty(n, dtype=np.uint32)
    pairs = np.empty(max(1, len(src)), dtype=np.uint64)
    c = _load().orc_lp_step(n, len(src), _p(src), _p(dst), _p(l_in), _p(l_out), _p(pairs))
    return l_out, int(c)


def pagerank(n, src, dst, damping=0.85, iters=20):
    """fp64 PageRank. Returns (rank f64[n], l1 per step f64[iters], dangling per step f64[iters])."""
    src, dst = _u32(src), _u32(dst)
    rank = np.empty(n, dtype=np.float64)
    l1 = np.zeros(max(iters, 1), dtype=np.float64)
    dang = np.zeros(max(iters, 1), dtype=np.float64)
    rc = _load().orc_pagerank(n, len(src), _p(src), _p(dst), damping, iters, _p(rank), _p(l1), _p(dang))
    if rc != 0:
        raise MemoryError("oracle pagerank allocation failed")
    return rank, l1[:iters].copy(), dang[:iters].copy()


def pagerank_step(n, src, dst, r_in, damping=0.85):
    """One fp64 superstep. Returns (r_out, dangling D of r_in, l1)."""
    src, dst = _u32(src), _u32(dst)
    r_in = np.ascontiguousarray(r_in, dtype=np.float64)
    outdeg = np.empty(n, dtype=np.uint64)
    _load().orc_outdeg(n, len(src), _p(src), _p(outdeg))
    r_out = np.empty(n, dtype=np.float64)
    l1 = C.c_double(0.0)
    d = _load().orc_pr_step(n, len(src), _p(src), _p(dst), _p(outdeg), damping, _p(r_in),
                            _p(r_out), C.addressof(l1))
    return r_out, float(d), float(l1.value)


def ppr(n, src, dst, source, damping=0.85, iters=20):
    """fp64 personalized PageRank from `source`."""
    src, dst = _u32(src), _u32(dst)
    rank = np.empty(n, dtype=np.float64)
    rc = _load().orc_ppr(n, len(src), _p(src), _p(dst), source, damping, iters, _p(rank))
    if rc != 0:
        raise ValueError("oracle ppr failed (allocation or source out of range)")
    return rank
