"""Failure detection under host-side fault injection (gxp_config.fault and the
GXP_FAULT environment variable).

Every fault here is made on the host: a device allocation that reports
out-of-memory, a host-to-device copy that is not enqueued, an exchange
between partitions whose kernels are not launched (a lost message), and, for
the allocation-free entry point (tests/test_zz_no_alloc.py) and the
persistent run's grid barrier, a bounded device wait that gives up at once. None of them faults, traps or hangs the
GPU. The tests check the exact status code, that a poisoning code leaves the
context answering GXP_E_STATE until gxp_destroy, that gxp_destroy is clean,
and that the context (allocation faults) or a fresh one (the others) then
computes the oracle's result.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2203_13005_gb300 import gxp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sssp_graph():
    wl = synth.SSSP_RMAT16.scaled(10)
    src, dst, w = wl.edges()
    d_ref, steps_ref, _ = oracle.sssp(wl.n_vertices, src, dst, w, 0)
    return wl.n_vertices, src, dst, w, d_ref, steps_ref


@pytest.fixture(scope="module")
def cc_graph():
    n = 1 << 11
    src, dst = synth.erdos_renyi(n, 1 << 11, 0x5EED)
    ref, steps, _ = oracle.cc(n, src, dst)
    return n, src, dst, ref, steps


def _sssp_run(ctx, g):
    n, src, dst, w, _, _ = g
    ctx.create_graph(n, 1)
    ctx.load_coo(src, dst, w)
    steps = ctx.run(gxp.GXP_ALGO_SSSP, source=0)
    return ctx.values(), steps


def _code(excinfo):
    return excinfo.value.code


def test_alloc_fault_every_allocation(gpu, sssp_graph):
    """The n-th device allocation fails (as an out-of-memory would): the call
    returns GXP_E_NOMEM, the context is not poisoned, and the same context
    then loads and runs the graph to the oracle's result."""
    d_ref, steps_ref = sssp_graph[4], sssp_graph[5]
    hit = 0
    for at in range(1, 200):
        ctx = gxp.Context(0, fault=gxp.GXP_FAULT_ALLOC, fault_at=at)
        try:
            try:
                d, steps = _sssp_run(ctx, sssp_graph)
            except gxp.GxpError as e:
                assert e.code == gxp.GXP_E_NOMEM, (at, e)
                hit += 1
                d, steps = _sssp_run(ctx, sssp_graph)   # retry on the same context
                assert np.array_equal(d, d_ref) and steps == steps_ref, at
                continue
            # past the last allocation of a run: nothing failed
            assert np.array_equal(d, d_ref) and steps == steps_ref
            break
        finally:
            ctx.close()
    else:
        pytest.fail("a run made 200 allocations or more")
    assert hit >= 5   # layout, values, stats and device-driven run buffers


def test_alloc_fault_then_new_context(gpu, sssp_graph):
    ctx = gxp.Context(0, fault=gxp.GXP_FAULT_ALLOC, fault_at=3)
    with pytest.raises(gxp.GxpError) as ei:
        _sssp_run(ctx, sssp_graph)
    assert _code(ei) == gxp.GXP_E_NOMEM
    ctx.close()
    with gxp.Context(0) as fresh:
        d, steps = _sssp_run(fresh, sssp_graph)
    assert np.array_equal(d, sssp_graph[4]) and steps == sssp_graph[5]


def _assert_poisoned(ctx, g):
    n, src, dst, w = g[:4]
    lib, h = ctx.lib, ctx.h
    t = gxp.TEMPLATES[gxp.GXP_ALGO_SSSP]
    out = np.empty(n, np.uint32)
    assert lib.gxp_create_graph(h, n, 1, None) == gxp.GXP_E_STATE
    assert lib.gxp_begin(h, gxp.GXP_ALGO_SSSP, 0, 0.85) == gxp.GXP_E_STATE
    assert lib.gxp_superstep(h, gxp.GXP_ALGO_SSSP, *t, None) == gxp.GXP_E_STATE
    assert lib.gxp_get_values(h, gxp.ALL_PARTS, out.ctypes.data, n) == gxp.GXP_E_STATE
    assert b"unusable" in lib.gxp_last_error(h)


def test_h2d_fault_poisons_until_destroy(gpu, sssp_graph):
    """The n-th host-to-device copy is not enqueued: GXP_E_CUDA, then
    GXP_E_STATE from every call until gxp_destroy; a fresh context works.
    Every copy of a load and run is tried in turn."""
    hit = 0
    for at in range(1, 100):
        ctx = gxp.Context(0, fault=gxp.GXP_FAULT_H2D, fault_at=at)
        try:
            try:
                d, steps = _sssp_run(ctx, sssp_graph)
            except gxp.GxpError as e:
                assert e.code == gxp.GXP_E_CUDA, (at, e)
                assert b"injected" in ctx.lib.gxp_last_error(ctx.h)
                _assert_poisoned(ctx, sssp_graph)
                hit += 1
                continue
            # past the last copy of a run: nothing failed
            assert np.array_equal(d, sssp_graph[4]) and steps == sssp_graph[5]
            break
        finally:
            ctx.close()
    else:
        pytest.fail("a run made 100 host-to-device copies or more")
    assert hit >= 4   # offsets, sources, weights, partition views, run control
    with gxp.Context(0) as fresh:
        d, steps = _sssp_run(fresh, sssp_graph)
    assert np.array_equal(d, sssp_graph[4]) and steps == sssp_graph[5]


def test_h2d_fault_from_environment(gpu, sssp_graph, monkeypatch):
    monkeypatch.setenv("GXP_FAULT", "h2d:2")
    ctx = gxp.Context(0)   # the environment is read when the context is made
    monkeypatch.delenv("GXP_FAULT")
    with pytest.raises(gxp.GxpError) as ei:
        _sssp_run(ctx, sssp_graph)
    assert _code(ei) == gxp.GXP_E_CUDA
    _assert_poisoned(ctx, sssp_graph)
    ctx.close()


@pytest.mark.parametrize("at", [1, 2, 4])
def test_dropped_exchange_is_detected(gpu, cc_graph, at):
    """The at-th exchange between partitions is dropped: the superstep's
    delivery mark is missing when its stats are read, so that superstep's
    call returns GXP_E_LOST and the context is poisoned. The supersteps before
    it match the oracle."""
    n, src, dst, ref, steps_ref = cc_graph
    assert steps_ref > at
    ctx = gxp.Context(0, fault=gxp.GXP_FAULT_SYNC_DROP, fault_at=at)
    ctx.create_graph(n, 4)
    ctx.load_coo(src, dst)
    ctx.begin(gxp.GXP_ALGO_CC)
    lab = np.arange(n, dtype=np.uint32)
    for t in range(1, at):
        ctx.superstep()
        lab, _ = oracle.cc_step(n, src, dst, lab)
        assert np.array_equal(ctx.values(), lab), t
    with pytest.raises(gxp.GxpError) as ei:
        ctx.superstep()
    assert _code(ei) == gxp.GXP_E_LOST
    assert ctx.lib.gxp_status_string(gxp.GXP_E_LOST) == b"GXP_E_LOST"
    _assert_poisoned(ctx, (n, src, dst, None))
    ctx.close()
    with gxp.Context(0) as fresh:
        fresh.create_graph(n, 4)
        fresh.load_coo(src, dst)
        assert fresh.run(gxp.GXP_ALGO_CC) == steps_ref
        assert np.array_equal(fresh.values(), ref)


def test_dropped_exchange_in_a_run(gpu, cc_graph):
    """gxp_run over partitions reads the stats once per chunk of supersteps:
    the drop is still reported, as GXP_E_LOST."""
    n, src, dst, _, _ = cc_graph
    ctx = gxp.Context(0, fault=gxp.GXP_FAULT_SYNC_DROP, fault_at=2)
    ctx.create_graph(n, 4)
    ctx.load_coo(src, dst)
    with pytest.raises(gxp.GxpError) as ei:
        ctx.run(gxp.GXP_ALGO_CC)
    assert _code(ei) == gxp.GXP_E_LOST
    ctx.close()


@pytest.mark.parametrize("algo", [gxp.GXP_ALGO_SSSP, gxp.GXP_ALGO_CC])
def test_persistent_run_barrier_gives_up(gpu, sssp_graph, algo):
    """A small single-partition run goes through the persistent kernel, whose
    CTAs meet at a bounded grid barrier after each superstep. With the
    timeout fault every barrier wait gives up at once (no wait runs out on
    its own): the run returns GXP_E_TIMEOUT, the context is poisoned, and a
    fresh context reaches the oracle's result through the same kernel."""
    n, src, dst, w, d_ref, steps_ref = sssp_graph
    ctx = gxp.Context(0, fault=gxp.GXP_FAULT_TIMEOUT)
    ctx.create_graph(n, 1)
    ctx.load_coo(src, dst, w)
    with pytest.raises(gxp.GxpError) as ei:
        ctx.run(algo, source=0)
    assert _code(ei) == gxp.GXP_E_TIMEOUT
    _assert_poisoned(ctx, sssp_graph)
    ctx.close()
    with gxp.Context(0) as fresh:
        d, steps = _sssp_run(fresh, sssp_graph)
        assert fresh.stats()["persistent_launches"] >= 1   # the same kernel, waits intact
    assert np.array_equal(d, d_ref) and steps == steps_ref


def test_persistent_batch_barrier_gives_up(gpu, sssp_graph):
    """The resident batched SSSP runs all its supersteps in one persistent
    kernel with a bounded grid barrier between them; under the timeout fault
    every barrier wait gives up at once: GXP_E_TIMEOUT, then GXP_E_STATE
    until gxp_destroy, and a fresh context's batch matches the oracle."""
    n, src, dst, w, d_ref, _ = sssp_graph
    sources = np.array([0, 1, 2], np.uint32)
    ctx = gxp.Context(0, fault=gxp.GXP_FAULT_TIMEOUT)
    ctx.create_graph(n, 1)
    ctx.load_coo(src, dst, w)
    with pytest.raises(gxp.GxpError) as ei:
        ctx.sssp_batch(sources)
    assert _code(ei) == gxp.GXP_E_TIMEOUT
    _assert_poisoned(ctx, sssp_graph)
    ctx.close()
    with gxp.Context(0) as fresh:
        fresh.create_graph(n, 1)
        fresh.load_coo(src, dst, w)
        dist, rep = fresh.sssp_batch(sources)
        assert rep["persistent"] == 1
    assert np.array_equal(dist[:, 0], d_ref)
    for j, s in enumerate(sources[1:], 1):
        ref, _, _ = oracle.sssp(n, src, dst, w, int(s))
        assert np.array_equal(dist[:, j], ref)


def test_unknown_fault_kinds_are_ignored(gpu, sssp_graph, monkeypatch):
    monkeypatch.setenv("GXP_FAULT", "nothing:3,alsonothing")
    with gxp.Context(0) as ctx:
        d, steps = _sssp_run(ctx, sssp_graph)
    assert np.array_equal(d, sssp_graph[4]) and steps == sssp_graph[5]
    assert os.environ.get("GXP_FAULT") == "nothing:3,alsonothing"
