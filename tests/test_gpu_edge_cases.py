"""Degenerate and ragged inputs through the C-ABI, against the oracle: empty
graphs, a single vertex, sizes one past the layout's window and warp
boundaries, long hub rows sorted in runs, and the same cases through the
query server."""
import numpy as np
import pytest

import oracle
from paper_2203_13005_gb300 import gxp, synth

pytestmark = pytest.mark.gpu

INF = gxp.INF


def _pr_close(r, ref):
    r = np.asarray(r, dtype=np.float64)
    assert np.all(np.abs(r - ref) <= 1e-4 * np.abs(ref) + 1e-12)
    assert np.abs(r - ref).sum() <= 1e-5


@pytest.mark.parametrize("keep_ids", [False, True])
@pytest.mark.parametrize("n", [1, 5])
def test_graph_without_edges(n, keep_ids):
    e = np.zeros(0, np.uint32)
    with gxp.Context(0, keep_ids=keep_ids) as c:
        c.create_graph(n, 1)
        c.load_coo(e, e, e)
        assert c.run(gxp.GXP_ALGO_SSSP, n - 1) == 1
        d = c.values()
        assert d[n - 1] == 0 and np.all(np.delete(d, n - 1) == INF)
        assert c.run(gxp.GXP_ALGO_CC) == 1
        assert np.array_equal(c.values(), np.arange(n, dtype=np.uint32))
        c.run(gxp.GXP_ALGO_PAGERANK, max_steps=20)
        _pr_close(c.values(), np.full(n, 1.0 / n))
        c.run(gxp.GXP_ALGO_PPR, 0, 0.85, 20)
        _pr_close(c.values(), np.eye(n)[0])


@pytest.mark.parametrize("n", [65537, 32 * 1000 + 7])
def test_ragged_sizes_across_windows(n):
    rng = np.random.default_rng(n)
    m = 6 * n
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    w = rng.integers(1, 50, m, dtype=np.uint32)
    d_ref, steps, _ = oracle.sssp(n, src, dst, w, 17)
    r_ref, _, _ = oracle.pagerank(n, src, dst, 0.85, 20)
    with gxp.Context(0) as c:
        c.create_graph(n, 1)
        c.load_coo(src, dst, w)
        assert c.run(gxp.GXP_ALGO_SSSP, 17) == steps
        assert np.array_equal(c.values(), d_ref)
        c.run(gxp.GXP_ALGO_PAGERANK, max_steps=20)
        _pr_close(c.values(), r_ref)


def test_long_hub_rows_sorted_in_runs():
    # two rows with 3 * 2048 + 5 and 2049 in-edges (runs of 2048 sorted apart),
    # plus a sparse random remainder; default tiles and small explicit ones
    rng = np.random.default_rng(5)
    n = 9000
    hub_a = rng.integers(0, n, 3 * 2048 + 5, dtype=np.uint32)
    hub_b = rng.integers(0, n, 2049, dtype=np.uint32)
    rest_s = rng.integers(0, n, 20000, dtype=np.uint32)
    rest_d = rng.integers(2, n, 20000, dtype=np.uint32)
    src = np.concatenate([hub_a, hub_b, rest_s])
    dst = np.concatenate([np.zeros(len(hub_a), np.uint32), np.ones(len(hub_b), np.uint32), rest_d])
    w = rng.integers(1, 9, len(src), dtype=np.uint32)
    d_ref, steps, _ = oracle.sssp(n, src, dst, w, 3)
    r_ref, _, _ = oracle.pagerank(n, src, dst, 0.85, 20)
    for tile, hub in ((0, 0), (2048, 1024), (300, 100)):
        with gxp.Context(0, tile_items=tile, hub_items=hub) as c:
            c.create_graph(n, 1)
            c.load_coo(src, dst, w)
            assert c.run(gxp.GXP_ALGO_SSSP, 3) == steps
            assert np.array_equal(c.values(), d_ref)
            c.run(gxp.GXP_ALGO_PAGERANK, max_steps=20)
            _pr_close(c.values(), r_ref)


def test_served_degenerate_graphs():
    e = np.zeros(0, np.uint32)
    ctx = gxp.Context(0)
    srv = gxp.Server(ctx)
    with ctx:
        srv.add_graph(1, e, e, e)                                  # one vertex, no edge
        srv.add_graph(3, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32),
                      np.array([4, 5], np.uint32))                  # a path 0 -> 1 -> 2
        srv.start()
        q0 = srv.submit(0, gxp.GXP_QUERY_SSSP, 0)
        q1 = srv.submit(0, gxp.GXP_QUERY_PPR, 0, 0.85, 20)
        q2 = srv.submit(1, gxp.GXP_QUERY_SSSP, 2)                  # source without out-edges
        q3 = srv.submit(1, gxp.GXP_QUERY_PPR, 0, 0.85, 3)
        assert np.array_equal(srv.result(q0, gxp.GXP_QUERY_SSSP, 0), [0])
        _pr_close(srv.result(q1, gxp.GXP_QUERY_PPR, 0), [1.0])
        assert np.array_equal(srv.result(q2, gxp.GXP_QUERY_SSSP, 1), [INF, INF, 0])
        _pr_close(srv.result(q3, gxp.GXP_QUERY_PPR, 1),
                  oracle.ppr(3, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), 0, 0.85, 3))
