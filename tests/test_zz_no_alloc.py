"""The allocation-free superstep entry point (gxp_superstep_min_noalloc).

It serves callers that cannot allocate device memory: its only scratch is a
fixed array inside the library, and every input and output comes from the
caller. This test drives it through the C-ABI with caller-owned device
buffers and checks two consecutive calls against the regular context path
(gxp_begin + gxp_superstep) and against the CPU oracle's superstep, bit for
bit as for every min-merge superstep; that repeated calls leave the device's
free memory unchanged; and that bad input is refused with a status code
before any edge block is staged. The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
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


def _call(algo, n, m, d_cp, d_src, d_w, d_cur, d_next):
    import torch
    lib = gxp.load()
    changed = C.c_uint64(0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.gxp_superstep_min_noalloc(algo, n, m, d_cp.data_ptr(), d_src.data_ptr(),
                                       None if d_w is None else d_w.data_ptr(), d_cur.data_ptr(),
                                       d_next.data_ptr(), C.byref(changed), stream)
    return rc, changed.value


def _noalloc(algo, n, m, d_cp, d_src, d_w, d_cur, d_next):
    rc, changed = _call(algo, n, m, d_cp, d_src, d_w, d_cur, d_next)
    assert rc == gxp.GXP_OK, gxp.load().gxp_status_string(rc)
    return changed


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
    # the oracle's Jacobi superstep, twice from the same start
    if algo == gxp.GXP_ALGO_SSSP:
        o1, oc1 = oracle.sssp_step(n, src, dst, w, cur)
        o2, oc2 = oracle.sssp_step(n, src, dst, w, o1)
    else:
        o1, oc1 = oracle.cc_step(n, src, dst, cur)
        o2, oc2 = oracle.cc_step(n, src, dst, o1)
    assert np.array_equal(got1, o1) and ch1 == oc1
    assert np.array_equal(got2, o2) and ch2 == oc2


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


def _small_cc(n=256, pairs=512, seed=7):
    src, dst = synth.erdos_renyi(n, pairs, seed)
    col_ptr, csrc, _ = _csc(n, src, dst, None)
    return n, src, dst, col_ptr, csrc


def test_noalloc_leaves_free_memory_unchanged():
    """Repeated calls allocate nothing: the device's free memory is the same
    before and after (the scratch is a static array of the library)."""
    import torch
    wl = synth.SSSP_RMAT16.scaled(12)
    src, dst, w = wl.edges()
    n = wl.n_vertices
    col_ptr, csrc, cw = _csc(n, src, dst, w)
    d_cp, d_src, d_w = _padded_device(col_ptr), _padded_device(csrc), _padded_device(cw)
    cur = np.full(n, gxp.INF, np.uint32)
    cur[0] = 0
    d_a = _padded_device(cur)
    d_b = torch.zeros_like(d_a)
    _noalloc(gxp.GXP_ALGO_SSSP, n, len(src), d_cp, d_src, d_w, d_a, d_b)   # first call: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(8):
        _noalloc(gxp.GXP_ALGO_SSSP, n, len(src), d_cp, d_src, d_w, d_a, d_b)
        _noalloc(gxp.GXP_ALGO_SSSP, n, len(src), d_cp, d_src, d_w, d_b, d_a)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_source_out_of_range_is_bounds():
    import torch
    n, src, dst, col_ptr, csrc = _small_cc()
    bad = csrc.copy()
    bad[len(bad) // 2] = n + 5
    d_cp, d_src = _padded_device(col_ptr), _padded_device(bad)
    d_a = _padded_device(np.arange(n, dtype=np.uint32))
    d_b = torch.zeros_like(d_a)
    rc, _ = _call(gxp.GXP_ALGO_CC, n, len(bad), d_cp, d_src, None, d_a, d_b)
    assert rc == gxp.GXP_E_BOUNDS
    # the next call with good input works: nothing is left behind
    d_good = _padded_device(csrc)
    rc, ch = _call(gxp.GXP_ALGO_CC, n, len(csrc), d_cp, d_good, None, d_a, d_b)
    assert rc == gxp.GXP_OK
    ref, rch = oracle.cc_step(n, src, dst, np.arange(n, dtype=np.uint32))
    assert np.array_equal(d_b[:n].cpu().numpy().view(np.uint32), ref) and ch == rch


@pytest.mark.parametrize("damage", ["decreasing", "first_not_zero", "last_not_n_edges"])
def test_noalloc_rejects_bad_offsets_before_staging(damage):
    """CSC offsets out of order are refused (GXP_E_INVAL) by the device-side
    check that runs before any edge block is cut or staged; d_next is not
    written."""
    import torch
    n, src, dst, col_ptr, csrc = _small_cc()
    cp = col_ptr.copy()
    if damage == "decreasing":
        cp[n // 2] = cp[n // 2 + 1] + 3   # a row whose end comes before its start
    elif damage == "first_not_zero":
        cp[0] = 1
    else:
        cp[n] = len(csrc) - 1
    d_cp, d_src = _padded_device(cp), _padded_device(csrc)
    d_a = _padded_device(np.arange(n, dtype=np.uint32))
    d_b = torch.full_like(d_a, 12345)
    rc, _ = _call(gxp.GXP_ALGO_CC, n, len(csrc), d_cp, d_src, None, d_a, d_b)
    assert rc == gxp.GXP_E_INVAL
    assert bool((d_b == 12345).all())


def test_noalloc_rejects_overlapping_values():
    import torch
    n, src, dst, col_ptr, csrc = _small_cc()
    d_cp, d_src = _padded_device(col_ptr), _padded_device(csrc)
    d_a = _padded_device(np.arange(2 * n, dtype=np.uint32))
    p = d_a.data_ptr()
    lib = gxp.load()
    s = torch.cuda.current_stream().cuda_stream
    for off in (0, 4, 4 * (n - 1)):
        assert lib.gxp_superstep_min_noalloc(gxp.GXP_ALGO_CC, n, len(csrc), d_cp.data_ptr(), d_src.data_ptr(),
                                             None, p, p + off, None, s) == gxp.GXP_E_INVAL
    # adjacent but disjoint ranges are fine
    assert lib.gxp_superstep_min_noalloc(gxp.GXP_ALGO_CC, n, len(csrc), d_cp.data_ptr(), d_src.data_ptr(),
                                         None, p, p + 4 * n, None, s) == gxp.GXP_OK


def test_noalloc_wait_that_gives_up_returns_timeout(monkeypatch):
    """GXP_FAULT=timeout makes every bounded wait on a bulk copy give up at
    once; each warp then waits for its own copies in flight and leaves. The
    call returns GXP_E_TIMEOUT, and the next call without the fault computes
    the oracle's superstep."""
    import torch
    wl = synth.SSSP_RMAT16.scaled(12)
    src, dst, w = wl.edges()
    n = wl.n_vertices
    col_ptr, csrc, cw = _csc(n, src, dst, w)
    d_cp, d_src, d_w = _padded_device(col_ptr), _padded_device(csrc), _padded_device(cw)
    cur = np.full(n, gxp.INF, np.uint32)
    cur[0] = 0
    d_a = _padded_device(cur)
    d_b = torch.zeros_like(d_a)
    monkeypatch.setenv("GXP_FAULT", "timeout")
    rc, _ = _call(gxp.GXP_ALGO_SSSP, n, len(src), d_cp, d_src, d_w, d_a, d_b)
    assert rc == gxp.GXP_E_TIMEOUT
    monkeypatch.delenv("GXP_FAULT")
    rc, ch = _call(gxp.GXP_ALGO_SSSP, n, len(src), d_cp, d_src, d_w, d_a, d_b)
    assert rc == gxp.GXP_OK
    ref, rch = oracle.sssp_step(n, src, dst, w, cur)
    assert np.array_equal(d_b[:n].cpu().numpy().view(np.uint32), ref) and ch == rch
