"""Synchronization caching under a budget (cache_slots): every partition's
LRU-weighted cache of remote copies (Section III-B2). At every superstep the
cached sets and the downloads follow the oracle's LRU trace (oracle/sync.py:
a copy enters when a superstep uses it, its weight decays by half and rises
with its reads, the lowest weights are evicted); values, changed counts,
upload lists and skip flags are the same at every budget."""
import numpy as np
import pytest

import oracle
from oracle import sync as osync
from paper_2203_13005_gb300 import gxp, synth

pytestmark = pytest.mark.gpu


def _graph(algo, n=3000, m=12000, seed=17):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    w = rng.integers(1, 60, m, dtype=np.uint32)
    if algo == "cc":
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
        w = None
    return n, src, dst, w


@pytest.mark.parametrize("budget", [0, 40, 1, 300, gxp.GXP_CACHE_NONE])
@pytest.mark.parametrize("algo", ["sssp", "cc"])
def test_lru_cache_follows_oracle(algo, budget):
    n, src, dst, w = _graph(algo)
    parts = 4
    b = [n * p // parts for p in range(parts + 1)]
    ref, steps, trace = osync.min_label_sync_trace(n, src, dst, b, algo, w=w, source=0)
    ghosts = osync.reads_per_copy(n, src, dst, b)
    cap = 0 if budget == gxp.GXP_CACHE_NONE else budget
    if budget != 0:
        lref, lsteps, trace0, ltrace = osync.lru_trace(n, src, dst, b, cap, algo, w=w, source=0)
        assert np.array_equal(lref, ref) and lsteps == steps
    with gxp.Context(0, cache_slots=budget) as c:
        c.create_graph(n, parts)
        c.load_coo(src, dst, w)
        c.begin(gxp.GXP_ALGO_SSSP if algo == "sssp" else gxp.GXP_ALGO_CC, 0)
        cum = 0
        for t in range(steps):
            c.superstep()
            uploads, skipped = trace[t]
            for p in range(parts):
                ids, vals, sk = c.sync(p)
                assert sk == skipped, (t, p)
                assert np.array_equal(ids, uploads[p][0]) and np.array_equal(vals, uploads[p][1]), (t, p)
            got = c.stats()["cache_downloads"]
            if budget == 0:
                assert got == 0
                for p in range(parts):
                    assert np.array_equal(c.cache(p), ghosts[p][0])
            else:
                cum += sum(trace0) if t == 0 else sum(d for _, d in ltrace[t - 1])
                assert got == cum, t
                for p in range(parts):
                    assert c.cache(p).tolist() == ltrace[t][p][0], (t, p)
        assert np.array_equal(c.values(), ref)


def test_lru_cache_with_lp_pagerank_and_runs():
    """Label propagation, PageRank and whole runs give the same values at
    every budget; a second gxp_begin starts from an empty cache again."""
    wl = synth.CC_ER24_P8.scaled(14)
    src, dst, _ = wl.edges()
    n = wl.n_vertices
    labels, steps, _ = oracle.lp(n, src, dst)
    cc_ref, cc_steps, _ = oracle.cc(n, src, dst)
    pr_ref, _, _ = oracle.pagerank(n, src, dst, 0.85, 20)
    b = [n * p // wl.parts for p in range(wl.parts + 1)]
    _, _, t0_500, _ = osync.lru_trace(n, src, dst, b, 500)
    for budget in (0, 500, gxp.GXP_CACHE_NONE):
        with gxp.Context(0, cache_slots=budget) as c:
            c.create_graph(n, wl.parts)
            c.load_coo(src, dst)
            assert c.run(gxp.GXP_ALGO_LP, max_steps=oracle.LP_MAX_STEPS) == steps
            assert np.array_equal(c.values(), labels)
            assert c.run(gxp.GXP_ALGO_CC) == cc_steps
            assert np.array_equal(c.values(), cc_ref)
            if budget == 0:
                assert c.stats()["cache_downloads"] == 0
            else:
                assert c.stats()["cache_downloads"] > 0
            c.run(gxp.GXP_ALGO_PAGERANK, max_steps=20)
            r = c.values().astype(np.float64)
            assert np.abs(r - pr_ref).sum() <= 1e-5
            assert np.max(np.abs(r - pr_ref) / pr_ref) <= 1e-4
            if budget == 500:
                # a fresh begin: the first superstep downloads what it uses into an empty cache
                c.begin(gxp.GXP_ALGO_CC)
                c.superstep()
                assert c.stats()["cache_downloads"] == sum(t0_500)


def test_cache_get_errors():
    n, src, dst, w = _graph("cc", 200, 400)
    with gxp.Context(0, cache_slots=8) as c:
        c.create_graph(n, 2)
        nn = gxp.C.c_uint64()
        assert c.lib.gxp_cache_get(c.h, 0, None, 0, gxp.C.byref(nn)) == gxp.GXP_E_STATE   # nothing loaded yet
        c.load_coo(src, dst)
        c.begin(gxp.GXP_ALGO_CC)
        assert c.lib.gxp_cache_get(c.h, 5, None, 0, gxp.C.byref(nn)) == gxp.GXP_E_INVAL
        assert c.lib.gxp_cache_get(c.h, 0, None, 0, None) == gxp.GXP_E_INVAL
        assert c.lib.gxp_cache_get(c.h, 0, None, 0, gxp.C.byref(nn)) == gxp.GXP_E_INVAL
        assert nn.value == 8
        assert len(c.cache(0)) == 8
