"""GPU parity: the CUDA superstep path (through the C-ABI) against the CPU oracle.

SSSP and CC are compared bit for bit (values, superstep counts, per-superstep
changed counts, and each partition's lazy-upload queue); PageRank within the
stated tolerance: per-vertex relative error <= 1e-4 and L1 <= 1e-5 against the
fp64 oracle. Edge blocks are forced small (1, 7, 31, 32, 33 merge items) so
hub splitting and the cross-tile combine run on small graphs too.
"""
import numpy as np
import pytest

import oracle
from oracle import sync as osync
from paper_2203_13005_gb300 import gxp, synth

pytestmark = pytest.mark.gpu

INF = gxp.INF
PR_REL, PR_L1 = 1e-4, 1e-5


def _ctx(n, parts=1, bounds=None, tile=0, hub=0, check=True):
    c = gxp.Context(0, tile_items=tile, hub_items=hub, check_bounds=check)
    c.create_graph(n, parts, bounds)
    return c


def _rand_graph(seed, n, m, wmax=100):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    w = rng.integers(1, wmax + 1, m, dtype=np.uint32)
    return src, dst, w


def _pr_check(r, r_ref):
    r = r.astype(np.float64)
    rel = np.abs(r - r_ref) / r_ref
    assert rel.max() <= PR_REL, f"max relative error {rel.max():.3g}"
    assert np.abs(r - r_ref).sum() <= PR_L1


# ---------------------------------------------------------------- SSSP

TILES = [(1, 0), (7, 3), (31, 8), (32, 16), (33, 1), (2048, 0)]


@pytest.mark.parametrize("tile,hub", TILES)
def test_sssp_clrs(tile, hub):
    e = np.array([[0, 1, 10], [0, 3, 5], [1, 2, 1], [1, 3, 2], [3, 1, 3], [3, 2, 9], [3, 4, 2],
                  [2, 4, 4], [4, 2, 6], [4, 0, 7]], dtype=np.uint32)
    with _ctx(5, tile=tile, hub=hub) as c:
        c.load_coo(e[:, 0], e[:, 1], e[:, 2])
        assert c.run(gxp.GXP_ALGO_SSSP, 0) == 4
        assert c.values().tolist() == [0, 8, 9, 5, 7]


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("tile,hub", TILES)
def test_sssp_random_stepwise(seed, tile, hub):
    n = [37, 200, 513, 1000][seed]
    src, dst, w = _rand_graph(seed, n, 4 * n)
    src[: n // 5] = dst[: n // 5]            # self-loops
    d_ref, steps_ref, ch_ref = oracle.sssp(n, src, dst, w, seed % n)
    with _ctx(n, tile=tile, hub=hub) as c:
        c.load_coo(src, dst, w)
        c.begin(gxp.GXP_ALGO_SSSP, seed % n)
        cur = np.full(n, INF, np.uint32)
        cur[seed % n] = 0
        for t in range(steps_ref):
            assert c.superstep() == ch_ref[t]
            nxt, _ = oracle.sssp_step(n, src, dst, w, cur)
            assert np.array_equal(c.values(), nxt)
            cur = nxt
        assert np.array_equal(c.values(), d_ref)


def test_sssp_rmat16_full():
    wl = synth.SSSP_RMAT16
    src, dst, w = wl.edges()
    d_ref, steps_ref, ch_ref = oracle.sssp(wl.n_vertices, src, dst, w, 0)
    with _ctx(wl.n_vertices) as c:
        c.load_coo(src, dst, w)
        steps = c.run(gxp.GXP_ALGO_SSSP, 0)
        assert steps == steps_ref
        assert np.array_equal(c.values(), d_ref)
        st = c.stats()
        assert st["supersteps"] == steps and st["last_changed"] == 0


def test_sssp_unreachable_and_empty():
    with _ctx(6) as c:
        c.load_coo(np.array([1, 2], np.uint32), np.array([2, 3], np.uint32), np.array([4, 5], np.uint32))
        assert c.run(gxp.GXP_ALGO_SSSP, 0) == 1
        assert c.values().tolist() == [0, INF, INF, INF, INF, INF]
        assert c.run(gxp.GXP_ALGO_SSSP, 1) == 3
        assert c.values().tolist() == [INF, 0, 4, 9, INF, INF]
    with _ctx(3) as c:
        c.load_coo(np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
        assert c.run(gxp.GXP_ALGO_SSSP, 2) == 1
        assert c.values().tolist() == [INF, INF, 0]


# ------------------------------------------------------------------ CC

def _undirected(seed, n, m):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, n, m, dtype=np.uint32)
    b = rng.integers(0, n, m, dtype=np.uint32)
    return np.concatenate([a, b]), np.concatenate([b, a])


@pytest.mark.parametrize("parts,bounds", [(1, None), (2, None), (3, [0, 0, 150, 400]), (8, None)])
@pytest.mark.parametrize("tile,hub", [(1, 0), (33, 1), (2048, 0)])
def test_cc_partitions_sync_trace(parts, bounds, tile, hub):
    n = 400
    src, dst = _undirected(11, n, 300)
    b = bounds if bounds is not None else [n * p // parts for p in range(parts + 1)]
    lab_ref, steps_ref, trace = osync.min_label_sync_trace(n, src, dst, b)
    with _ctx(n, parts, bounds, tile=tile, hub=hub) as c:
        c.load_coo(src, dst)
        c.begin(gxp.GXP_ALGO_CC)
        for t in range(steps_ref):
            c.superstep()
            uploads, skipped = trace[t]
            for p in range(parts):
                ids, vals, sk = c.sync(p)
                assert sk == skipped
                assert np.array_equal(ids, uploads[p][0]), (t, p)
                assert np.array_equal(vals, uploads[p][1]), (t, p)
        assert np.array_equal(c.values(), lab_ref)
        st = c.stats()
        if parts > 1:
            assert st["syncs_skipped"] == sum(s for _, s in trace)
            assert st["syncs_done"] + st["syncs_skipped"] == steps_ref


@pytest.mark.parametrize("p_cross", [1e-3, 1e-4])
def test_sssp_clustered_graph_skips_syncs(p_cross):
    # communities on the partitions with few pairs between them: the
    # supersteps that change no boundary vertex skip their exchange, and the
    # uploads and skip flags follow the sync oracle superstep for superstep
    import dataclasses
    wl = dataclasses.replace(synth.SSSP_CLUSTERED24_P8.scaled(14), p_cross=p_cross)
    src, dst, w = wl.edges()
    n = wl.n_vertices
    b = [n * p // wl.parts for p in range(wl.parts + 1)]
    d_ref, steps_ref, trace = osync.min_label_sync_trace(n, src, dst, b, "sssp", w=w, source=0)
    assert sum(s for _, s in trace) >= 2   # skipping triggers on this graph
    with _ctx(n, wl.parts, None) as c:
        c.load_coo(src, dst, w)
        c.begin(gxp.GXP_ALGO_SSSP, 0)
        for t in range(steps_ref):
            c.superstep()
            uploads, skipped = trace[t]
            for p in range(wl.parts):
                ids, vals, sk = c.sync(p)
                assert sk == skipped, (t, p)
                assert np.array_equal(ids, uploads[p][0]), (t, p)
                assert np.array_equal(vals, uploads[p][1]), (t, p)
        assert np.array_equal(c.values(), d_ref)
        assert c.run(gxp.GXP_ALGO_SSSP, 0) == steps_ref
        st = c.stats()
        assert st["syncs_skipped"] == sum(s for _, s in trace)
        assert st["syncs_done"] + st["syncs_skipped"] == steps_ref


def test_cc_disconnected_partitions_always_skip():
    a = [(u, v) for u in range(4) for v in range(4) if u != v]
    e = np.array(a + [(u + 4, v + 4) for u, v in a], dtype=np.uint32)
    with _ctx(8, 2) as c:
        c.load_coo(e[:, 0], e[:, 1])
        steps = c.run(gxp.GXP_ALGO_CC)
        assert c.values().tolist() == [0] * 4 + [4] * 4
        st = c.stats()
        assert st["syncs_done"] == 0 and st["syncs_skipped"] == steps


def test_cc_er_scaled_one_vs_eight_partitions():
    wl = synth.CC_ER24_P8.scaled(18)
    src, dst, _ = wl.edges()
    n = wl.n_vertices
    lab_ref, steps_ref, _ = oracle.cc(n, src, dst)
    res = []
    for parts in (1, 8):
        with _ctx(n, parts) as c:
            c.load_coo(src, dst)
            steps = c.run(gxp.GXP_ALGO_CC)
            assert steps == steps_ref
            res.append(c.values())
    assert np.array_equal(res[0], lab_ref) and np.array_equal(res[1], lab_ref)


@pytest.mark.slow
def test_cc_er24_8parts_full():
    wl = synth.CC_ER24_P8
    src, dst, _ = wl.edges()
    n = wl.n_vertices
    lab_ref, steps_ref, _ = oracle.cc(n, src, dst)
    with _ctx(n, wl.parts) as c:
        c.load_coo(src, dst)
        steps = c.run(gxp.GXP_ALGO_CC)
        assert steps == steps_ref
        assert np.array_equal(c.values(), lab_ref)


# ------------------------------------------------------------- PageRank

@pytest.mark.parametrize("tile,hub", TILES)
def test_pagerank_rmat_small_tiles(tile, hub):
    src, dst = synth.rmat(10, 1 << 14, 21)
    n = 1 << 10
    r_ref, _, _ = oracle.pagerank(n, src, dst, 0.85, 20)
    with _ctx(n, tile=tile, hub=hub) as c:
        c.load_coo(src, dst)
        assert c.run(gxp.GXP_ALGO_PAGERANK, damping=0.85, max_steps=20) == 20
        _pr_check(c.values(), r_ref)


def test_pagerank_stepwise_sums():
    # the exact fixed-point sums (dangling mass, L1 delta) against the fp64
    # oracle, superstep by superstep; fp32 ranks leave an ulp-level floor of
    # about N * 2^-24 * max(r) on the L1 delta
    src, dst = synth.rmat(11, 1 << 15, 22)
    n = 1 << 11
    outdeg = np.bincount(src, minlength=n)
    r = np.full(n, 1.0 / n)
    with _ctx(n, tile=64, hub=16) as c:
        c.load_coo(src, dst)
        c.begin(gxp.GXP_ALGO_PAGERANK, damping=0.85)
        for t in range(8):
            c.superstep()
            r_next, _, l1 = oracle.pagerank_step(n, src, dst, r, 0.85)
            st = c.stats()
            floor = n * 2.0**-24 * r_next.max()
            assert abs(st["last_l1_delta"] - l1) <= 1e-3 * l1 + floor, t
            assert st["last_dangling"] == pytest.approx(float(r_next[outdeg == 0].sum()), rel=1e-5)
            _pr_check(c.values(), r_next)
            r = r_next


def test_pagerank_hub_in_star_many_tiles():
    k = 50_000                                   # in-degree far above a tile
    n = k + 1
    src = np.arange(1, n, dtype=np.uint32)
    dst = np.zeros(k, np.uint32)
    r_ref, _, _ = oracle.pagerank(n, src, dst, 0.85, 20)
    with _ctx(n) as c:
        c.load_coo(src, dst)
        c.run(gxp.GXP_ALGO_PAGERANK, damping=0.85, max_steps=20)
        _pr_check(c.values(), r_ref)
    with _ctx(n) as c:                           # same hub through the min path
        c.load_coo(src, dst, np.full(k, 3, np.uint32))
        c.run(gxp.GXP_ALGO_SSSP, 7)
        d = c.values()
        assert d[7] == 0 and d[0] == 3 and np.sum(d == INF) == n - 2


def test_pagerank_degenerate():
    with _ctx(4) as c:                           # no edges: every vertex dangling
        c.load_coo(np.zeros(0, np.uint32), np.zeros(0, np.uint32))
        c.run(gxp.GXP_ALGO_PAGERANK, damping=0.85, max_steps=20)
        assert np.allclose(c.values(), 0.25, rtol=1e-6)
    with _ctx(1) as c:                           # one vertex with a self-loop
        c.load_coo(np.zeros(1, np.uint32), np.zeros(1, np.uint32))
        c.run(gxp.GXP_ALGO_PAGERANK, damping=0.85, max_steps=20)
        assert c.values()[0] == pytest.approx(1.0, rel=1e-6)


@pytest.mark.parametrize("n_zero", [1, 32, 32 * 5 + 7, 32 * 9 + 31])
@pytest.mark.parametrize("keep", [False, True])
def test_pagerank_rows_without_in_edges(n_zero, keep):
    # the slices of rows without in-edges are applied several per warp: ragged
    # group counts, pad rows in the last slice, and personalized PageRank from
    # a source that has no in-edges
    rng = np.random.default_rng(n_zero + 17 * keep)
    k = 300                                        # vertices with in-edges
    n = k + n_zero
    m = 4000
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, k, m, dtype=np.uint32)
    r_ref, _, _ = oracle.pagerank(n, src, dst, 0.85, 20)
    s = n - 1                                      # no in-edges
    p_ref = oracle.ppr(n, src, dst, s, 0.85, 20)
    with gxp.Context(0, keep_ids=keep, check_bounds=True) as c:
        c.create_graph(n, 1)
        c.load_coo(src, dst)
        c.run(gxp.GXP_ALGO_PAGERANK, damping=0.85, max_steps=20)
        _pr_check(c.values(), r_ref)
        c.run(gxp.GXP_ALGO_PPR, s, 0.85, 20)
        p = c.values().astype(np.float64)
        assert np.all(np.abs(p - p_ref) <= 1e-4 * p_ref + 1e-9)


def test_reloads_reuse_device_memory():
    # the context keeps freed device memory in its pool: graphs of different
    # sizes loaded one after another into one context, each run checked
    # against the oracle, and the same graph twice holds the same bytes
    held = {}
    with gxp.Context(0) as c:
        for scale, seed in [(12, 1), (10, 2), (13, 3), (12, 1)]:
            src, dst = synth.rmat(scale, 16 << scale, seed)
            n = 1 << scale
            r_ref, _, _ = oracle.pagerank(n, src, dst, 0.85, 20)
            lab_ref, steps_ref, _ = oracle.cc(n, src, dst)
            c.create_graph(n, 1)
            c.load_coo(src, dst)
            c.run(gxp.GXP_ALGO_PAGERANK, damping=0.85, max_steps=20)
            _pr_check(c.values(), r_ref)
            assert c.run(gxp.GXP_ALGO_CC) == steps_ref
            assert np.array_equal(c.values(), lab_ref)
            b = c.stats()["device_bytes"]
            assert held.setdefault((scale, seed), b) == b


def test_partitioned_then_single_partition_graph():
    # one context: a graph in 4 partitions (exchange buffers), then graphs in
    # one partition (none), then partitions again, each against the oracle
    with gxp.Context(0, check_bounds=True) as c:
        for parts, scale, seed in [(4, 11, 5), (1, 12, 6), (1, 10, 7), (4, 12, 8)]:
            n = 1 << scale
            src, dst = synth.erdos_renyi(n, 4 << scale, seed)
            lab_ref, steps_ref, _ = oracle.cc(n, src, dst)
            c.create_graph(n, parts)
            c.load_coo(src, dst)
            assert c.run(gxp.GXP_ALGO_CC) == steps_ref, (parts, scale)
            assert np.array_equal(c.values(), lab_ref), (parts, scale)


def test_pagerank_rmat22_full_and_deterministic():
    wl = synth.PAGERANK_RMAT22
    src, dst, _ = wl.edges()
    n = wl.n_vertices
    r_ref, l1_ref, dang_ref = oracle.pagerank(n, src, dst, 0.85, 20)
    with _ctx(n, check=False) as c:
        c.load_coo(src, dst)
        c.run(gxp.GXP_ALGO_PAGERANK, damping=0.85, max_steps=20)
        r1 = c.values()
        st = c.stats()
        c.run(gxp.GXP_ALGO_PAGERANK, damping=0.85, max_steps=20)
        r2 = c.values()
    _pr_check(r1, r_ref)
    assert np.array_equal(r1.view(np.uint32), r2.view(np.uint32))
    # the mass stays 1 to within fp32 rounding of the ranks (the global sums are exact)
    assert abs(float(r1.astype(np.float64).sum()) - 1.0) <= 1e-6
    assert st["last_dangling"] == pytest.approx(
        float(r_ref[np.bincount(src, minlength=n) == 0].sum()), rel=1e-5)


# ------------------------------------------------------- formats / API

def test_formats_and_device_inputs_agree():
    import torch
    src, dst, w = _rand_graph(5, 300, 2000)
    n = 300
    d_ref, steps_ref, _ = oracle.sssp(n, src, dst, w, 3)
    order = np.argsort(dst, kind="stable")
    col_ptr = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(dst, minlength=n), out=col_ptr[1:])
    rorder = np.argsort(src, kind="stable")
    row_ptr = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    loads = {
        "coo": (gxp.GXP_FMT_COO, src, dst, w),
        "csc": (gxp.GXP_FMT_CSC, col_ptr, np.ascontiguousarray(src[order]), np.ascontiguousarray(w[order])),
        "csr": (gxp.GXP_FMT_CSR, row_ptr, np.ascontiguousarray(dst[rorder]), np.ascontiguousarray(w[rorder])),
        "coo_device": (gxp.GXP_FMT_COO, torch.from_numpy(src.astype(np.int32)).cuda(),
                       torch.from_numpy(dst.astype(np.int32)).cuda(), torch.from_numpy(w.astype(np.int32)).cuda()),
    }
    for name, (fmt, a, b, ww) in loads.items():
        with _ctx(n) as c:
            c.load_partition(0, fmt, len(src), a, b, ww)
            assert c.run(gxp.GXP_ALGO_SSSP, 3) == steps_ref, name
            assert np.array_equal(c.values(), d_ref), name


def test_csc_single_partition_loads_on_device():
    """A single-partition CSC goes straight to device memory (host or device
    arrays) and is checked there; the batched path still works on it."""
    import torch
    n = 400
    src, dst, w = _rand_graph(6, n, 3000)
    order = np.argsort(dst, kind="stable")
    col_ptr = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(dst, minlength=n), out=col_ptr[1:])
    s_sorted, w_sorted = np.ascontiguousarray(src[order]), np.ascontiguousarray(w[order])
    d_ref, steps_ref, _ = oracle.sssp(n, src, dst, w, 5)
    d_ref7, _, _ = oracle.sssp(n, src, dst, w, 7)
    variants = {
        "host": (col_ptr, s_sorted, w_sorted),
        "device": (torch.from_numpy(col_ptr.view(np.int64)).cuda(), torch.from_numpy(s_sorted.view(np.int32)).cuda(),
                   torch.from_numpy(w_sorted.view(np.int32)).cuda()),
    }
    for name, (a, b, ww) in variants.items():
        with _ctx(n) as c:
            c.load_partition(0, gxp.GXP_FMT_CSC, len(src), a, b, ww)
            assert c.run(gxp.GXP_ALGO_SSSP, 5) == steps_ref, name
            assert np.array_equal(c.values(), d_ref), name
            dist, _ = c.sssp_batch(np.array([5, 7], np.uint32))
            assert np.array_equal(dist[:, 0], d_ref) and np.array_equal(dist[:, 1], d_ref7), name
            c.load_partition(0, gxp.GXP_FMT_CSC, len(src), a, b, ww)   # reload replaces it
            assert c.run(gxp.GXP_ALGO_SSSP, 7) >= 1
            assert np.array_equal(c.values(), d_ref7), name
    k = int(np.argmax(np.diff(col_ptr.astype(np.int64)) > 0))
    decreasing = col_ptr.copy()
    decreasing[k + 1] = decreasing[k] - 1 if decreasing[k] > 0 else 0
    decreasing[k] = col_ptr[k + 1]
    bad_end = col_ptr.copy()
    bad_end[n] += 1
    bad_src = s_sorted.copy()
    bad_src[len(src) // 2] = n
    with _ctx(n) as c:
        for cp, sv in ((decreasing, s_sorted), (bad_end, s_sorted), (col_ptr, bad_src)):
            with pytest.raises(gxp.GxpError) as ei:
                c.load_partition(0, gxp.GXP_FMT_CSC, len(src), cp, sv, w_sorted)
            assert ei.value.code == gxp.GXP_E_INVAL
        c.load_partition(0, gxp.GXP_FMT_CSC, len(src), col_ptr, s_sorted, w_sorted)   # still usable
        c.run(gxp.GXP_ALGO_SSSP, 5)
        assert np.array_equal(c.values(), d_ref)


@pytest.mark.parametrize("parts", [1, 3])
def test_run_stops_at_first_quiet_superstep(parts):
    """gxp_run enqueues supersteps in chunks; the ones after the first quiet
    superstep return at once on the device and are rolled back."""
    n = 500
    src, dst, w = _rand_graph(9, n, 4000)
    d_ref, steps_ref, _ = oracle.sssp(n, src, dst, w, 1)
    with _ctx(n, parts=parts) as c:
        c.load_coo(src, dst, w)
        assert c.run(gxp.GXP_ALGO_SSSP, 1) == steps_ref
        st = c.stats()
        assert st["supersteps"] == steps_ref and st["last_changed"] == 0
        assert np.array_equal(c.values(), d_ref)
        assert c.superstep() == 0                      # continuing from the fixed point
        assert np.array_equal(c.values(), d_ref)
        assert c.stats()["supersteps"] == steps_ref + 1
        assert c.run(gxp.GXP_ALGO_SSSP, 1, max_steps=2) == 2
        assert c.run(gxp.GXP_ALGO_CC) >= 1
        labels, _, _ = oracle.cc(n, src, dst)
        assert np.array_equal(c.values(), labels)


def test_relabelled_and_input_order_agree():
    """A single partition is renumbered by in-degree inside the engine unless
    keep_ids is set; results come back in input ids either way."""
    wl = synth.SSSP_RMAT16.scaled(12)
    src, dst, w = wl.edges()
    n = wl.n_vertices
    d_ref, steps_ref, _ = oracle.sssp(n, src, dst, w, 3)
    labels_ref, _, _ = oracle.cc(n, np.concatenate([src, dst]), np.concatenate([dst, src]))
    r_ref, _, _ = oracle.pagerank(n, src, dst, 0.85, 20)
    out = {}
    for keep in (False, True):
        with gxp.Context(0, keep_ids=keep) as c:
            c.create_graph(n, 1)
            c.load_coo(src, dst, w)
            assert c.run(gxp.GXP_ALGO_SSSP, 3) == steps_ref
            assert np.array_equal(c.values(), d_ref)
            d_mid = c.values()
            c.set_values(d_mid)                         # checkpoint round trip through the mapping
            assert c.superstep() == 0 and np.array_equal(c.values(), d_ref)
            c.run(gxp.GXP_ALGO_PAGERANK, max_steps=20)
            out[keep] = c.values().copy()
            _pr_check(out[keep], r_ref)
        with gxp.Context(0, keep_ids=keep) as c:
            c.create_graph(n, 1)
            c.load_coo(np.concatenate([src, dst]), np.concatenate([dst, src]))
            c.run(gxp.GXP_ALGO_CC)
            assert np.array_equal(c.values(), labels_ref)


def test_errors_are_status_codes():
    with _ctx(4) as c:
        with pytest.raises(gxp.GxpError) as ei:
            c.superstep(gxp.GXP_ALGO_CC)
        assert ei.value.code == gxp.GXP_E_STATE
        with pytest.raises(gxp.GxpError) as ei:
            c.load_coo(np.array([0], np.uint32), np.array([9], np.uint32))
        assert ei.value.code == gxp.GXP_E_INVAL
        c.load_coo(np.array([0, 1], np.uint32), np.array([1, 2], np.uint32))
        with pytest.raises(gxp.GxpError) as ei:
            c.begin(gxp.GXP_ALGO_SSSP, 0)                   # no weights
        assert ei.value.code == gxp.GXP_E_INVAL
        c.begin(gxp.GXP_ALGO_CC)
        with pytest.raises(gxp.GxpError) as ei:
            c.superstep(gxp.GXP_ALGO_CC, template=(gxp.GXP_GEN_CONTRIB, gxp.GXP_MERGE_SUM, gxp.GXP_APPLY_MIN))
        assert ei.value.code == gxp.GXP_E_UNSUPPORTED
        assert c.superstep() == 2                           # context still usable
        with pytest.raises(gxp.GxpError) as ei:
            c.sync(7)
        assert ei.value.code == gxp.GXP_E_INVAL


def test_checkpoint_resume_bit_identical():
    wl = synth.SSSP_RMAT16.scaled(12)
    src, dst, w = wl.edges()
    n = wl.n_vertices
    d_ref, steps_ref, _ = oracle.sssp(n, src, dst, w, 0)
    k = steps_ref // 2
    with _ctx(n, 4) as c:
        c.load_coo(src, dst, w)
        c.begin(gxp.GXP_ALGO_SSSP, 0)
        for _ in range(k):
            c.superstep()
        snap = c.values().copy()
    with _ctx(n, 4) as c:
        c.load_coo(src, dst, w)
        c.begin(gxp.GXP_ALGO_SSSP, 0)
        c.set_values(snap)
        t = k
        while c.superstep() != 0:
            t += 1
        assert t + 1 == steps_ref
        assert np.array_equal(c.values(), d_ref)
