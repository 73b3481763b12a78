"""The allocation-free superstep entry point (gxp_superstep_min_noalloc).

It serves callers that cannot allocate device memory: its only scratch is a
fixed array inside the library, and every input and output comes from the
caller. This test drives it through the C-ABI with caller-owned device
buffers and checks two consecutive calls against the regular context path
(gxp_begin + gxp_superstep), bit for bit as for every min-merge superstep.
The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2203_13005_gb300 import gxp, synth

pytestmark = pytest.mark.gpu


def _padded_device(a: np.ndarray):
    """uint32 device copy of `a`, 16-byte aligned, readable to round_up(len, 4) + 4."""
    import torch
    n = (len(a) + 3) // 4 * 4 + 4
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    if len(a):
        t[: len(a)] = torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()
    assert t.data_ptr() % 16 == 0
    return t


def _csc(n, src, dst, w):
    order = np.argsort(dst, kind="stable")
    col_ptr = np.zeros(n + 1, np.uint32)
    np.cumsum(np.bincount(dst, minlength=n), out=col_ptr[1:])
    return col_ptr, src[order], (None if w is None else w[order])


def _noalloc(algo, n, m, d_cp, d_src, d_w, d_cur, d_next):
    import torch
    lib = gxp.load()
    changed = C.c_uint64(0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.gxp_superstep_min_noalloc(algo, n, m, d_cp.data_ptr(), d_src.data_ptr(),
                                       None if d_w is None else d_w.data_ptr(), d_cur.data_ptr(),
                                       d_next.data_ptr(), C.byref(changed), stream)
    assert rc == gxp.GXP_OK, lib.gxp_status_string(rc)
    return changed.value


def _two_calls_match_context(algo, n, src, dst, w, source=0):
    import torch
    col_ptr, csrc, cw = _csc(n, src, dst, w)
    d_cp, d_src = _padded_device(col_ptr), _padded_device(csrc)
    d_w = None if cw is None else _padded_device(cw)
    if algo == gxp.GXP_ALGO_SSSP:
        cur = np.full(n, gxp.INF, np.uint32)
        cur[source] = 0
    else:
        cur = np.arange(n, dtype=np.uint32)
    d_a = _padded_device(cur)
    d_b = torch.zeros_like(d_a)
    d_c = torch.zeros_like(d_a)
    ch1 = _noalloc(algo, n, len(src), d_cp, d_src, d_w, d_a, d_b)
    ch2 = _noalloc(algo, n, len(src), d_cp, d_src, d_w, d_b, d_c)
    got1 = d_b[:n].cpu().numpy().view(np.uint32)
    got2 = d_c[:n].cpu().numpy().view(np.uint32)
    with gxp.Context(0) as ctx:
        ctx.create_graph(n, 1)
        ctx.load_coo(src, dst, w)
        ctx.begin(algo, source)
        ref_ch1 = ctx.superstep()
        ref1 = ctx.values().copy()
        ref_ch2 = ctx.superstep()
        ref2 = ctx.values().copy()
    assert np.array_equal(got1, ref1) and ch1 == ref_ch1
    assert np.array_equal(got2, ref2) and ch2 == ref_ch2
    assert ch1 > 0


def test_noalloc_sssp_two_calls_match_superstep():
    wl = synth.SSSP_RMAT16.scaled(14)
    src, dst, w = wl.edges()
    _two_calls_match_context(gxp.GXP_ALGO_SSSP, wl.n_vertices, src, dst, w)


def test_noalloc_cc_two_calls_match_superstep():
    src, dst = synth.erdos_renyi(1 << 14, 1 << 15, 5)
    _two_calls_match_context(gxp.GXP_ALGO_CC, 1 << 14, src, dst, None)


def test_noalloc_rejects_oversized_and_misaligned():
    import torch
    lib = gxp.load()
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    # beyond the fixed scratch: n_vertices + n_edges > 2^28 (rejected before any device access)
    assert lib.gxp_superstep_min_noalloc(gxp.GXP_ALGO_CC, 1 << 27, 1 << 28, p, p, None, p, p, None,
                                         None) == gxp.GXP_E_INVAL
    # misaligned CSC pointer
    assert lib.gxp_superstep_min_noalloc(gxp.GXP_ALGO_CC, 4, 4, p + 4, p, None, p, p, None,
                                         None) == gxp.GXP_E_INVAL
    # PageRank is not a min-merge template
    assert lib.gxp_superstep_min_noalloc(gxp.GXP_ALGO_PAGERANK, 4, 4, p, p, None, p, p, None,
                                         None) == gxp.GXP_E_UNSUPPORTED
