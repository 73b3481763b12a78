"""GPU tests of personalized PageRank and of the query server.

* The single-query PPR path (gxp_run(GXP_ALGO_PPR)) and every served PPR
  query are held to the PageRank tolerance against the fp64 oracle
  (per-vertex relative error <= 1e-4 where the oracle is non-zero, exact zeros
  where it is zero, L1 <= 1e-5); served SSSP queries are bit-exact.
* A query's result is the same bit for bit alone and in a mix of other
  queries that arrive while it runs (continuous batching).
* Admission by slot and by result memory, stop / restart, and the error codes.
"""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2203_13005_gb300 import gxp, synth

pytestmark = pytest.mark.gpu

PR_REL, PR_L1 = 1e-4, 1e-5
SSSP, PPR = gxp.GXP_QUERY_SSSP, gxp.GXP_QUERY_PPR


def _ppr_check(r, r_ref):
    r = np.asarray(r, dtype=np.float64)
    zero = r_ref == 0.0
    assert np.all(r[zero] == 0.0), "non-zero rank where the oracle has none"
    rel = np.abs(r[~zero] - r_ref[~zero]) / r_ref[~zero]
    assert rel.max() <= PR_REL, f"max relative error {rel.max():.3g}"
    assert np.abs(r - r_ref).sum() <= PR_L1


def _graph(scale, i=0):
    wl = synth.SERVE_GRAPHS[i].scaled(scale)
    src, dst, w = wl.edges()
    return wl.n_vertices, src, dst, w


@pytest.fixture(scope="module")
def graphs():
    return [_graph(11, 0), _graph(12, 1)]


def _server(graphs, weighted=(True, True), **start):
    ctx = gxp.Context(0)
    srv = gxp.Server(ctx)
    for (n, src, dst, w), wt in zip(graphs, weighted):
        srv.add_graph(n, src, dst, w if wt else None)
    srv.start(**start)
    return ctx, srv


def _sources(n, src, k, seed):
    return synth.sources_with_out_edges(n, src, k, seed)


# ------------------------------------------------------ single-query PPR

@pytest.mark.parametrize("tile,hub", [(2048, 0), (7, 3)])
def test_engine_ppr_vs_oracle(graphs, tile, hub):
    n, src, dst, w = graphs[1]
    for s in _sources(n, src, 3, 11):
        with gxp.Context(0, tile_items=tile, hub_items=hub) as c:
            c.create_graph(n, 1)
            c.load_coo(src, dst)
            steps = c.run(gxp.GXP_ALGO_PPR, int(s), 0.85, 20)
            assert steps == 20
            _ppr_check(c.values(), oracle.ppr(n, src, dst, int(s), 0.85, 20))


def test_engine_ppr_partitions_and_dangling_source():
    # in-star: the leaves point at the centre, which has no out-edge (dangling)
    k = 40
    src = np.arange(1, k + 1, dtype=np.uint32)
    dst = np.zeros(k, dtype=np.uint32)
    n = k + 1
    for s in (0, 7):
        ref = oracle.ppr(n, src, dst, s, 0.85, 20)
        with gxp.Context(0) as c:
            c.create_graph(n, 3)
            c.load_coo(src, dst)
            c.run(gxp.GXP_ALGO_PPR, s, 0.85, 20)
            _ppr_check(c.values(), ref)


# ---------------------------------------------------------------- serving

def test_served_queries_match_oracle(graphs):
    ctx, srv = _server(graphs)
    with ctx:
        jobs = []
        for gi, (n, src, dst, w) in enumerate(graphs):
            for j, s in enumerate(_sources(n, src, 12, 100 + gi)):
                kind = SSSP if j % 2 == 0 else PPR
                d = 0.85 if j % 4 != 1 else 0.5
                it = 20 if j % 4 != 3 else 7
                jobs.append((srv.submit(gi, kind, int(s), d, it), gi, kind, int(s), d, it))
        for q, gi, kind, s, d, it in jobs:
            n, src, dst, w = graphs[gi]
            info = srv.info(q)
            res = srv.result(q, kind, gi)
            if kind == SSSP:
                ref, _, _ = oracle.sssp(n, src, dst, w, s)
                assert np.array_equal(res, ref), f"sssp graph {gi} source {s}"
            else:
                assert info["state"] in (gxp.GXP_QUERY_RUNNING, gxp.GXP_QUERY_DONE, gxp.GXP_QUERY_QUEUED)
                _ppr_check(res, oracle.ppr(n, src, dst, s, d, it))
        rep = srv.report()
        assert rep["completed"] == len(jobs) and rep["failed"] == 0 and rep["queued"] == 0


def test_alone_and_in_the_mix_bit_identical(graphs):
    """The same query, first alone on an idle server, then in the middle of a
    stream of other queries that keep arriving (and being collected) while it
    runs."""
    n, src, dst, w = graphs[1]
    probe = int(_sources(n, src, 2, 7)[0])
    others = _sources(n, src, 150, 8)
    ctx, srv = _server(graphs)
    with ctx:
        alone = {}
        for kind in (SSSP, PPR):
            q = srv.submit(1, kind, probe, 0.85, 20)
            alone[kind] = srv.result(q, kind, 1)
            assert srv.report()["running"] == 0

        lock = threading.Lock()   # submit + record are atomic with respect to the collector
        probe_ids, feeder_ids = {}, set()
        stop = threading.Event()
        stats = {"query_supersteps": 0, "collected": 0}

        def feeder():   # keeps the lanes busy before, during and after the probe
            for k in range(len(others)):
                for gi in (0, 1):
                    with lock:
                        feeder_ids.add(srv.submit(gi, SSSP if k % 2 else PPR,
                                                  int(others[k]) % graphs[gi][0], 0.85, 20))
                if stop.is_set():
                    break

        def collector():   # releases the feeder's results so admission never starves
            buf = np.empty(max(srv.n), dtype=np.uint32)
            while True:
                q = srv.next_done(200)
                if q == 0:
                    if stop.is_set():
                        return
                    continue
                with lock:
                    mine = q in feeder_ids
                if mine:
                    stats["query_supersteps"] += srv.info(q)["supersteps"]
                    srv.poll(q, buf)
                    stats["collected"] += 1

        tf, tc = threading.Thread(target=feeder), threading.Thread(target=collector)
        tf.start()
        tc.start()
        t0 = time.monotonic()
        while srv.report()["running"] < 8 and time.monotonic() - t0 < 10.0:
            time.sleep(0.0005)
        assert srv.report()["running"] >= 8
        for kind in (SSSP, PPR):
            with lock:
                probe_ids[kind] = srv.submit(1, kind, probe, 0.85, 20)
        mixed = {kind: srv.result(probe_ids[kind], kind, 1) for kind in (SSSP, PPR)}
        running_after = srv.report()["running"]
        tf.join()
        while srv.report()["queued"] + srv.report()["running"] > 0:
            time.sleep(0.01)
        stop.set()
        tc.join()
        rep = srv.report()
        for kind in (SSSP, PPR):
            assert np.array_equal(alone[kind].view(np.uint32), mixed[kind].view(np.uint32)), kind
        # others were still running after the probes finished, and the lanes
        # shared supersteps: more query-supersteps than lane supersteps
        assert running_after > 0 or rep["queued"] > 0 or stats["collected"] > 0
        assert stats["collected"] == len(feeder_ids)
        assert stats["query_supersteps"] > rep["sssp_supersteps"] + rep["ppr_supersteps"]
    ref, _, _ = oracle.sssp(n, src, dst, w, probe)
    assert np.array_equal(mixed[SSSP], ref)
    _ppr_check(mixed[PPR], oracle.ppr(n, src, dst, probe, 0.85, 20))


def test_one_slot_server_same_results(graphs):
    n, src, dst, w = graphs[0]
    srcs = _sources(n, src, 4, 21)
    out = {}
    for slots in (1, 64):
        ctx, srv = _server(graphs, max_slots=slots)
        with ctx:
            qs = [(srv.submit(0, k, int(s), 0.85, 20), k) for s in srcs for k in (SSSP, PPR)]
            out[slots] = [srv.result(q, k, 0) for q, k in qs]
    for a, b in zip(out[1], out[64]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_admission_waits_for_result_memory(graphs):
    n, src, dst, w = graphs[0]
    srcs = _sources(n, src, 6, 31)
    ctx, srv = _server(graphs, results_per_graph=2)
    with ctx:
        qs = [srv.submit(0, PPR, int(s), 0.85, 5) for s in srcs]
        done = [srv.next_done(10000), srv.next_done(10000)]
        assert sorted(done) == qs[:2]
        assert srv.next_done(300) == 0   # nobody collected: nothing else may be admitted
        rep = srv.report()
        assert rep["completed"] == 2 and rep["running"] == 0 and rep["queued"] == 4
        assert srv.info(qs[2])["state"] == gxp.GXP_QUERY_QUEUED
        buf = np.empty(n, dtype=np.float32)
        assert srv.poll(qs[0], buf)      # frees one result buffer -> one more admitted
        assert srv.next_done(10000) == qs[2]
        for q in qs[1:]:
            assert srv.poll(q, buf)
        assert srv.report()["completed"] == 6


def test_stop_fails_waiting_queries_and_restart(graphs):
    n, src, dst, w = graphs[0]
    srcs = _sources(n, src, 4, 41)
    ctx, srv = _server(graphs, results_per_graph=1)
    with ctx:
        qs = [srv.submit(0, SSSP, int(s)) for s in srcs]
        assert srv.next_done(10000) == qs[0]
        srv.stop()
        for q in qs[1:]:
            with pytest.raises(gxp.GxpError) as ei:
                srv.poll(q, np.empty(n, dtype=np.uint32))
            assert ei.value.code == gxp.GXP_E_STATE
        res0 = srv.result(qs[0], SSSP, 0)   # done before the stop: still collectable
        srv.start()
        q = srv.submit(0, SSSP, int(srcs[0]))
        assert np.array_equal(srv.result(q, SSSP, 0), res0)
        ref, _, _ = oracle.sssp(n, src, dst, w, int(srcs[0]))
        assert np.array_equal(res0, ref)


def test_serving_errors(graphs):
    n, src, dst, w = graphs[0]
    ctx = gxp.Context(0)
    srv = gxp.Server(ctx)
    with ctx:
        with pytest.raises(gxp.GxpError) as ei:
            srv.submit(0, SSSP, 0)
        assert ei.value.code == gxp.GXP_E_STATE
        with pytest.raises(gxp.GxpError) as ei:
            srv.add_graph(n, src, np.full_like(dst, n), w)
        assert ei.value.code == gxp.GXP_E_INVAL
        srv.add_graph(n, src, dst, w)
        srv.add_graph(n, src, dst, None)     # PPR only
        srv.start(queue_cap=4)
        with pytest.raises(gxp.GxpError) as ei:
            srv.add_graph(n, src, dst, w)
        assert ei.value.code == gxp.GXP_E_STATE
        for args, code in [((2, SSSP, 0), gxp.GXP_E_INVAL), ((0, 5, 0), gxp.GXP_E_INVAL),
                           ((0, SSSP, n), gxp.GXP_E_INVAL), ((0, PPR, 0, 1.0), gxp.GXP_E_INVAL),
                           ((1, SSSP, 0), gxp.GXP_E_UNSUPPORTED)]:
            with pytest.raises(gxp.GxpError) as ei:
                srv.submit(*args)
            assert ei.value.code == code, args
        with pytest.raises(gxp.GxpError) as ei:
            srv.poll(12345, None, 0)
        assert ei.value.code == gxp.GXP_E_INVAL
        q = srv.submit(1, PPR, 0, 0.85, 3)
        assert srv.poll(q, None, -1)         # done, not released
        with pytest.raises(gxp.GxpError) as ei:
            srv.poll(q, np.empty(n - 1, dtype=np.float32))
        assert ei.value.code == gxp.GXP_E_INVAL
        assert srv.poll(q, np.empty(n, dtype=np.float32))
        with pytest.raises(gxp.GxpError):
            srv.poll(q, None, 0)             # released
        # queue capacity: with one slot and one result buffer per graph busy, the queue fills
        srv.stop()
        srv.start(max_slots=1, results_per_graph=1, queue_cap=2)
        held = srv.submit(1, PPR, 0, 0.85, 2)
        assert srv.next_done(10000) == held  # its result buffer stays held
        srv.submit(1, PPR, 1, 0.85, 2)
        srv.submit(1, PPR, 2, 0.85, 2)
        with pytest.raises(gxp.GxpError) as ei:
            srv.submit(1, PPR, 3, 0.85, 2)
        assert ei.value.code == gxp.GXP_E_BUSY


def test_device_output_buffer(graphs):
    torch = pytest.importorskip("torch")
    n, src, dst, w = graphs[0]
    s = int(_sources(n, src, 1, 51)[0])
    ctx, srv = _server(graphs)
    with ctx:
        q = srv.submit(0, SSSP, s)
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        assert srv.poll(q, out)
        ref, _, _ = oracle.sssp(n, src, dst, w, s)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)


def test_served_sssp_wide_weights():
    # weights above 255: the server keeps 8-byte edges for this graph
    rng = np.random.default_rng(78)
    n, m = 2000, 30000
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    w = rng.integers(1, 70000, m, dtype=np.uint32)
    ctx = gxp.Context(0)
    srv = gxp.Server(ctx)
    with ctx:
        srv.add_graph(n, src, dst, w)
        srv.start()
        srcs = _sources(n, src, 6, 3)
        qs = [srv.submit(0, SSSP, int(s)) for s in srcs]
        for q, s in zip(qs, srcs):
            ref, _, _ = oracle.sssp(n, src, dst, w, int(s))
            assert np.array_equal(srv.result(q, SSSP, 0), ref)
